// Batched ensemble: many independent 2-D meshes of different sizes and
// orders advanced together, one persistent launch per SSPRK(4,3) stage.
//
// Work items are tiles (EPB consecutive elements) of any member; CTAs of a
// persistent grid take items from an atomic counter, copy the member's
// kernel arguments to shared memory and run the same tile code as the
// single-mesh stage kernel (stage_block), specialised by the member's order.
// One step (counter resets + four stage launches) is captured once in a CUDA
// graph and replayed.  Members are independent, so there is no exchange
// between them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "dg_ctx.h"

using namespace dgm;

namespace {

constexpr int kEnsThreads = 256;

struct EnsMember {
    KArgs<float> args;   // mesh, reference tables, derived / base / table / flag pointers
    float *U[2];         // U^n, work stage
    float *trace[2];
    float g_half, g_sixth;
    double fall_w[4];    // the stages' weights in the step for the rain fall-out
    int K, rain;
    int tiles;           // element tiles of this member
};

template <int K, bool RAIN>
struct EnsShape : Shape<2, K, RAIN, 256> {};

template <class S>
constexpr size_t ens_smem() { return stage_smem_bytes<S, float>(); }

constexpr size_t max2(size_t a, size_t b) { return a > b ? a : b; }

constexpr size_t kEnsSmem =
    max2(max2(max2(ens_smem<EnsShape<1, true>>(), ens_smem<EnsShape<2, true>>()),
              max2(ens_smem<EnsShape<3, true>>(), ens_smem<EnsShape<4, true>>())),
         max2(ens_smem<EnsShape<5, true>>(),
              max2(max2(ens_smem<EnsShape<1, false>>(), ens_smem<EnsShape<2, false>>()),
                   max2(max2(ens_smem<EnsShape<3, false>>(), ens_smem<EnsShape<4, false>>()),
                        ens_smem<EnsShape<5, false>>()))));

// reference-element tables per order (identical for all members of one order)
__constant__ RefData<float> c_ens_ref[5];

template <int K, bool RAIN>
__device__ __noinline__ void ens_tile(const KArgs<float> &A, int tile, unsigned char *smem) {
    static_assert(EnsShape<K, RAIN>::NT == kEnsThreads, "2-D tiles use 256 threads for every order");
    stage_block<EnsShape<K, RAIN>, float, MODE_STAGE>(A, c_ens_ref[K - 1], tile, smem);
}

// MINB: CTAs per SM the register budget is sized for (2: 128 registers per
// thread, 3: 80); one of the autotuner's knobs.
// An item is up to tiles_per_item consecutive element tiles of one member
// (items[i] = (member, first tile)).
template <int MINB>
__global__ void __launch_bounds__(kEnsThreads, MINB) k_ens_stage(const EnsMember *members,
                                                             const int2 *items, int n_items,
                                                             int tiles_per_item, int stage,
                                                             unsigned int *counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ KArgs<float> s_args;
    __shared__ int s_item, s_k, s_rain, s_member;
    if (threadIdx.x == 0) s_member = -1;
    // work queue, not a wait: every pass takes the next item from a counter
    // that only grows, so a CTA leaves after at most n_items + 1 passes
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int2 wi = items[it];
        const EnsMember *m = members + wi.x;
        // the member's arguments stay in shared memory while the CTA's items
        // belong to the same member (s_member was set before the last barrier)
        const bool fresh = wi.x != s_member;
        if (fresh) {
            const int *src = reinterpret_cast<const int *>(&m->args);
            int *dst = reinterpret_cast<int *>(&s_args);
            for (int i = threadIdx.x; i < (int)(sizeof(KArgs<float>) / sizeof(int)); i += blockDim.x)
                dst[i] = src[i];
        }
        __syncthreads();
        if (threadIdx.x == 0 && fresh) {
            s_member = wi.x;
            // SSPRK(4,3) Shu-Osher stages; the traces of U^n sit in trace[0] at each step start
            float *Un = m->U[0], *Uw = m->U[1];
            switch (stage) {
                case 0: s_args.Uin = Un; s_args.Un = Un; s_args.Uout = Uw;
                        s_args.alpha = 0.0f; s_args.beta = 1.0f; s_args.gdt = m->g_half;
                        s_args.trace_in = m->trace[0]; s_args.trace_out = m->trace[1]; break;
                case 1: s_args.Uin = Uw; s_args.Un = Uw; s_args.Uout = Uw;
                        s_args.alpha = 0.0f; s_args.beta = 1.0f; s_args.gdt = m->g_half;
                        s_args.trace_in = m->trace[1]; s_args.trace_out = m->trace[0]; break;
                case 2: s_args.Uin = Uw; s_args.Un = Un; s_args.Uout = Uw;
                        s_args.alpha = (float)(2.0 / 3.0); s_args.beta = (float)(1.0 / 3.0);
                        s_args.gdt = m->g_sixth;
                        s_args.trace_in = m->trace[0]; s_args.trace_out = m->trace[1]; break;
                default: s_args.Uin = Uw; s_args.Un = Uw; s_args.Uout = Un;
                         s_args.alpha = 0.0f; s_args.beta = 1.0f; s_args.gdt = m->g_half;
                         s_args.trace_in = m->trace[1]; s_args.trace_out = m->trace[0]; break;
            }
            s_args.fall_w = m->fall_w[stage];
            s_k = m->K;
            s_rain = m->rain;
        }
        __syncthreads();
        const int t_end = min(wi.y + tiles_per_item, m->tiles);
        for (int tile = wi.y; tile < t_end; ++tile) {
            if (s_rain) {
                switch (s_k) {
                    case 1: ens_tile<1, true>(s_args, tile, smem_raw); break;
                    case 2: ens_tile<2, true>(s_args, tile, smem_raw); break;
                    case 3: ens_tile<3, true>(s_args, tile, smem_raw); break;
                    case 4: ens_tile<4, true>(s_args, tile, smem_raw); break;
                    default: ens_tile<5, true>(s_args, tile, smem_raw); break;
                }
            } else {
                switch (s_k) {
                    case 1: ens_tile<1, false>(s_args, tile, smem_raw); break;
                    case 2: ens_tile<2, false>(s_args, tile, smem_raw); break;
                    case 3: ens_tile<3, false>(s_args, tile, smem_raw); break;
                    case 4: ens_tile<4, false>(s_args, tile, smem_raw); break;
                    default: ens_tile<5, false>(s_args, tile, smem_raw); break;
                }
            }
            __syncthreads();
        }
    }
}

int epb_of(int K, int rain) {
    switch (K) {
        case 1: return rain ? EnsShape<1, true>::EPB : EnsShape<1, false>::EPB;
        case 2: return rain ? EnsShape<2, true>::EPB : EnsShape<2, false>::EPB;
        case 3: return rain ? EnsShape<3, true>::EPB : EnsShape<3, false>::EPB;
        case 4: return rain ? EnsShape<4, true>::EPB : EnsShape<4, false>::EPB;
        default: return rain ? EnsShape<5, true>::EPB : EnsShape<5, false>::EPB;
    }
}

}  // namespace

struct dg_ensemble {
    int n = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<dg_ctx *> members;
    std::vector<double> dt;
    std::vector<int> tiles;          // tiles per member
    EnsMember *d_members = nullptr;
    int2 *d_items = nullptr;
    int n_items = 0;
    unsigned int *d_counters = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    int blocks_per_sm = 2;
    int item_order = 1;
    int regs = 0;                    // 0: k_ens_stage<2>, 1: k_ens_stage<3>
    int tiles_per_item = 1;
    int sm_count = 0;
    int grid = 0;
    long long dofs = 0;
    int lanes = 0;                   // > 0: the branch schedule with this many lanes
};

namespace {

void destroy_graph(dg_ensemble *E) {
    if (E->exec) cudaGraphExecDestroy(E->exec);
    if (E->graph) cudaGraphDestroy(E->graph);
    E->exec = nullptr;
    E->graph = nullptr;
}

// Upload the member table and the item list (order: 0 member-major,
// 1 round-robin over members, 2 largest members first); capture one step.
int build(dg_ensemble *E) {
    destroy_graph(E);
    std::vector<EnsMember> h(E->n);
    for (int i = 0; i < E->n; ++i) {
        dg_ctx *c = E->members[i];
        EnsMember &m = h[i];
        std::memset(&m, 0, sizeof(m));
        KArgs<float> &A = m.args;
        A.M = c->M;
        A.ref = c->ref32;
        A.derived = (float *)c->derived;
        A.bnode = (const float *)c->bnode_r;
        A.bface = (const float *)c->bface_r;
        A.bnode_d = c->bnode_d;
        A.rvs_tab = c->rvs_tab;
        A.bsplit = c->bsplit;
        A.flags = c->flags;
        A.fallout = c->fallout;
        for (int s = 0; s < 3; ++s) m.fall_w[s] = E->dt[i] / 6.0;
        m.fall_w[3] = 0.5 * E->dt[i];
        m.U[0] = (float *)c->U[0];
        m.U[1] = (float *)c->U[1];
        m.trace[0] = (float *)c->trace[0];
        m.trace[1] = (float *)c->trace[1];
        m.g_half = (float)(0.5 * E->dt[i]);
        m.g_sixth = (float)(E->dt[i] / 6.0);
        m.K = c->cfg.order;
        m.rain = c->cfg.rain;
        m.tiles = E->tiles[i];
    }
    {
        RefData<float> refs[5];
        std::memset(refs, 0, sizeof(refs));
        for (int i = 0; i < E->n; ++i) refs[E->members[i]->cfg.order - 1] = E->members[i]->ref32;
        if (cudaMemcpyToSymbolAsync(c_ens_ref, refs, sizeof(refs), 0, cudaMemcpyHostToDevice,
                                    E->stream) != cudaSuccess)
            return DG_ECUDA;
    }
    std::vector<int2> items;
    std::vector<int> order(E->n);
    for (int i = 0; i < E->n; ++i) order[i] = i;
    if (E->item_order == 2)
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return E->members[a]->nodes > E->members[b]->nodes;
        });
    const int tpi = E->tiles_per_item;
    if (E->item_order == 1) {
        int maxt = 0;
        for (int i = 0; i < E->n; ++i) maxt = std::max(maxt, E->tiles[i]);
        for (int t = 0; t < maxt; t += tpi)
            for (int i : order)
                if (t < E->tiles[i]) items.push_back(make_int2(i, t));
    } else {
        for (int i : order)
            for (int t = 0; t < E->tiles[i]; t += tpi) items.push_back(make_int2(i, t));
    }
    E->n_items = (int)items.size();
    if (E->d_members) cudaFree(E->d_members);
    if (E->d_items) cudaFree(E->d_items);
    E->d_members = nullptr;
    E->d_items = nullptr;
    if (cudaMalloc(&E->d_members, sizeof(EnsMember) * E->n) != cudaSuccess) return DG_ENOMEM;
    if (cudaMalloc(&E->d_items, sizeof(int2) * items.size()) != cudaSuccess) return DG_ENOMEM;
    if (cudaMemcpyAsync(E->d_members, h.data(), sizeof(EnsMember) * E->n, cudaMemcpyHostToDevice,
                        E->stream) != cudaSuccess)
        return DG_ECUDA;
    if (cudaMemcpyAsync(E->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice,
                        E->stream) != cudaSuccess)
        return DG_ECUDA;
    if (cudaStreamSynchronize(E->stream) != cudaSuccess) return DG_ECUDA;

    auto kern = E->regs ? k_ens_stage<3> : k_ens_stage<2>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEnsSmem) !=
        cudaSuccess)
        return DG_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kEnsThreads, kEnsSmem) !=
        cudaSuccess)
        return DG_ECUDA;
    const int bps = std::max(1, std::min(E->blocks_per_sm, per_sm));
    const int grid = bps * E->sm_count;
    E->grid = grid;

    if (cudaStreamBeginCapture(E->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return DG_ECUDA;
    cudaError_t err = cudaMemsetAsync(E->d_counters, 0, 4 * sizeof(unsigned int), E->stream);
    for (int s = 0; s < 4 && err == cudaSuccess; ++s) {
        kern<<<grid, kEnsThreads, kEnsSmem, E->stream>>>(E->d_members, E->d_items, E->n_items,
                                                         E->tiles_per_item, s, E->d_counters + s);
        err = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    const cudaError_t end = cudaStreamEndCapture(E->stream, &g);
    if (err != cudaSuccess || end != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return DG_ECUDA;
    }
    E->graph = g;
    if (cudaGraphInstantiate(&E->exec, g, 0) != cudaSuccess) return DG_ECUDA;
    return DG_OK;
}

// Branch schedule: member i's step is dg_step_async on its own context (the
// single-mesh face pass and stage kernels), issued on lane l(i); the lanes
// are parallel branches of one captured graph, so members of different
// lanes run concurrently and members of one lane one after another.
// Members go, largest first, to the lane with the fewest DOFs so far.
int build_branches(dg_ensemble *E, int lanes) {
    destroy_graph(E);
    lanes = std::max(1, std::min(lanes, E->n));
    std::vector<int> order(E->n);
    for (int i = 0; i < E->n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return E->members[a]->nodes * E->members[a]->nf > E->members[b]->nodes * E->members[b]->nf;
    });
    std::vector<long long> load(lanes, 0);
    std::vector<std::vector<int>> lane(lanes);
    for (int i : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lane[l].push_back(i);
        load[l] += E->members[i]->nodes * E->members[i]->nf;
    }
    std::vector<cudaStream_t> ls(lanes, nullptr);
    std::vector<cudaEvent_t> join(lanes, nullptr);
    cudaEvent_t fork = nullptr;
    int st = DG_OK;
    for (int l = 0; l < lanes && st == DG_OK; ++l) {
        if (cudaStreamCreateWithFlags(&ls[l], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&join[l], cudaEventDisableTiming) != cudaSuccess)
            st = DG_ECUDA;
    }
    if (st == DG_OK && cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) st = DG_ECUDA;
    // relaxed capture: a member's first launch of a kernel sets its
    // shared-memory attribute, which is not a stream operation
    bool capturing = false;
    if (st == DG_OK) {
        if (cudaStreamBeginCapture(E->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) st = DG_ECUDA;
        else capturing = true;
    }
    if (st == DG_OK && cudaEventRecord(fork, E->stream) != cudaSuccess) st = DG_ECUDA;
    for (int l = 0; l < lanes && st == DG_OK; ++l) {
        if (cudaStreamWaitEvent(ls[l], fork, 0) != cudaSuccess) {
            st = DG_ECUDA;
            break;
        }
        for (int i : lane[l]) {
            dg_ctx *c = E->members[i];
            const cudaStream_t own = c->stream;
            c->stream = ls[l];
            st = dg_step_async(c, E->dt[i], 1);
            c->stream = own;
            if (st != DG_OK) break;
        }
        if (st == DG_OK && (cudaEventRecord(join[l], ls[l]) != cudaSuccess ||
                            cudaStreamWaitEvent(E->stream, join[l], 0) != cudaSuccess))
            st = DG_ECUDA;
    }
    cudaGraph_t g = nullptr;
    if (capturing) {
        const cudaError_t end = cudaStreamEndCapture(E->stream, &g);
        if (st == DG_OK && end != cudaSuccess) st = DG_ECUDA;
    }
    if (st == DG_OK) {
        E->graph = g;
        g = nullptr;
        if (cudaGraphInstantiate(&E->exec, E->graph, 0) != cudaSuccess) st = DG_ECUDA;
    }
    if (g) cudaGraphDestroy(g);
    if (fork) cudaEventDestroy(fork);
    for (int l = 0; l < lanes; ++l) {
        if (join[l]) cudaEventDestroy(join[l]);
        if (ls[l]) cudaStreamDestroy(ls[l]);
    }
    if (st != DG_OK) {
        destroy_graph(E);
        return st;
    }
    E->lanes = lanes;
    E->grid = lanes;
    E->n_items = E->n;
    return DG_OK;
}

// dt[i] and, for every member, its split and traces of U^n in trace buffer 0
int set_dt_and_prepare(dg_ensemble *E, const double *dt) {
    for (int i = 0; i < E->n; ++i)
        if (!(dt[i] > 0.0)) return DG_EINVAL;
    for (int i = 0; i < E->n; ++i) E->dt[i] = dt[i];
    for (dg_ctx *c : E->members) {
        if (!c->derived_valid || c->parity != 0) {
            const int st = ctx_prepare(c, c->U[0], 0);
            if (st != DG_OK) return st;
            c->parity = 0;
            c->derived_valid = true;
        }
    }
    return DG_OK;
}

}  // namespace

extern "C" {

int dg_ensemble_create(dg_ensemble **out, int n, const dg_config *cfgs, const dg_bubble *bubbles,
                       void *cuda_stream) {
    if (!out || n < 1 || !cfgs || !bubbles) return DG_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (cfgs[i].dim != 2 || (cfgs[i].precision != DG_FP32_BULK && cfgs[i].precision != DG_FP32_PERT))
            return DG_EINVAL;
    dg_ensemble *E = new (std::nothrow) dg_ensemble();
    if (!E) return DG_ENOMEM;
    E->n = n;
    cudaGetDevice(&E->device);
    cudaDeviceGetAttribute(&E->sm_count, cudaDevAttrMultiProcessorCount, E->device);
    if (cuda_stream) {
        E->stream = (cudaStream_t)cuda_stream;
    } else {
        // graph capture needs a stream other than the legacy default stream
        if (cudaStreamCreateWithFlags(&E->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete E;
            return DG_ECUDA;
        }
        E->own_stream = true;
    }
    int st = DG_OK;
    for (int i = 0; i < n && st == DG_OK; ++i) {
        dg_ctx *c = nullptr;
        st = dg_init_mesh(&c, &cfgs[i], E->stream);
        if (st == DG_OK) {
            c->in_ensemble = true;
            E->members.push_back(c);
            st = dg_init_bubble(c, &bubbles[i], nullptr, DG_HOST);
        }
        if (st == DG_OK) {
            E->tiles.push_back((int)((c->ne + epb_of(c->cfg.order, c->cfg.rain) - 1) /
                                     epb_of(c->cfg.order, c->cfg.rain)));
            E->dofs += c->nodes * c->nf;
        }
    }
    if (st == DG_OK && cudaMalloc(&E->d_counters, 4 * sizeof(unsigned int)) != cudaSuccess) st = DG_ENOMEM;
    if (st != DG_OK) {
        dg_ensemble_free(E);
        return st;
    }
    E->dt.assign(n, 0.0);
    *out = E;
    return DG_OK;
}

void dg_ensemble_free(dg_ensemble *E) {
    if (!E) return;
    cudaStreamSynchronize(E->stream);
    destroy_graph(E);
    for (dg_ctx *c : E->members) dg_free(c);
    if (E->d_members) cudaFree(E->d_members);
    if (E->d_items) cudaFree(E->d_items);
    if (E->d_counters) cudaFree(E->d_counters);
    if (E->own_stream) cudaStreamDestroy(E->stream);
    delete E;
}

int dg_ensemble_member(dg_ensemble *E, int i, dg_ctx **ctx) {
    if (!E || !ctx || i < 0 || i >= E->n) return DG_EINVAL;
    *ctx = E->members[i];
    return DG_OK;
}

long long dg_ensemble_dofs(const dg_ensemble *E) { return E ? E->dofs : 0; }

int dg_ensemble_launch_shape(const dg_ensemble *E, int *grid, int *n_items) {
    if (!E || !grid || !n_items) return DG_EINVAL;
    *grid = E->grid;
    *n_items = E->n_items;
    return DG_OK;
}

int dg_ensemble_configure(dg_ensemble *E, const double *dt, int blocks_per_sm, int item_order,
                          int regs, int tiles_per_item) {
    if (!E || !dt || blocks_per_sm < 1 || item_order < 0 || item_order > 2) return DG_EINVAL;
    if (regs != 0 && regs != 1) return DG_EINVAL;
    if (tiles_per_item < 1 || tiles_per_item > 64) return DG_EINVAL;
    const int st = set_dt_and_prepare(E, dt);
    if (st != DG_OK) return st;
    E->regs = regs;
    E->tiles_per_item = tiles_per_item;
    E->blocks_per_sm = blocks_per_sm;
    E->item_order = item_order;
    E->lanes = 0;
    return build(E);
}

int dg_ensemble_configure_branches(dg_ensemble *E, const double *dt, int lanes) {
    if (!E || !dt || lanes < 1) return DG_EINVAL;
    for (dg_ctx *c : E->members)
        if (!c->face_pass) return DG_EINVAL;
    const int st = set_dt_and_prepare(E, dt);
    if (st != DG_OK) return st;
    const int bs = build_branches(E, lanes);
    if (bs != DG_OK) return bs;
    return cudaStreamSynchronize(E->stream) == cudaSuccess ? DG_OK : DG_ECUDA;
}

int dg_ensemble_step_async(dg_ensemble *E, int nsteps) {
    if (!E || nsteps < 0) return DG_EINVAL;
    if (!E->exec) return DG_ESTATE;
    for (int s = 0; s < nsteps; ++s)
        if (cudaGraphLaunch(E->exec, E->stream) != cudaSuccess) return DG_ECUDA;
    return DG_OK;
}

int dg_ensemble_step(dg_ensemble *E, int nsteps) {
    int st = dg_ensemble_step_async(E, nsteps);
    if (st != DG_OK) return st;
    int worst = DG_OK;
    for (dg_ctx *c : E->members) {
        const int s = dg_check_status(c, nullptr);
        if (s == DG_ECUDA) return s;
        if (s == DG_ENONPHYS || (s == DG_ENOCONV && worst == DG_OK)) worst = s;
    }
    return worst;
}

}  // extern "C"
