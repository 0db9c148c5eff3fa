// C interface of the moist DG library (declared in include/dgmoist.h).
//
// Host side: validation, reference-element tables, buffers, the stage
// schedule of SSPRK(4,3) and the hydrostatic column of the warm-bubble
// workload.  Every step of the right-hand side and of the time step runs in
// the CUDA kernels of dg_device.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "dg_launch.cuh"
#include "dgmoist.h"

using namespace dgm;

namespace {

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = (cudaSetDevice(dev) == cudaSuccess);
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

// ---- reference element -----------------------------------------------------
// Gauss-Legendre points: roots of P_n by Newton's method (three-term
// recurrence for P_n and its derivative), weights 2 / ((1 - x^2) P_n'(x)^2).
void legendre_pd(int n, double x, double &p, double &dp) {
    double p0 = 1.0, p1 = x;
    if (n == 0) {
        p = 1.0;
        dp = 0.0;
        return;
    }
    for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    p = p1;
    dp = n * (p0 - x * p1) / (1.0 - x * x);
}

void gauss_rule(int n, double *x, double *w) {
    for (int i = 0; i < n; ++i) {
        double t = -std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre_pd(n, t, p, dp);
            const double dt = p / dp;
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        double p, dp;
        legendre_pd(n, t, p, dp);
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

// Lagrange basis through x[0..n): value at s; derivative matrix by the
// barycentric formula D[i][a] = l_a'(x_i).
double lagrange_at(const double *x, int n, int a, double s) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
        if (m != a) v *= (s - x[m]) / (x[a] - x[m]);
    return v;
}

// l_a'(s) = l_a(s) sum_{m != a} 1 / (s - x_m), for s not a node (s = +-1 here)
double lagrange_deriv_at(const double *x, int n, int a, double s) {
    double sum = 0.0;
    for (int m = 0; m < n; ++m)
        if (m != a) sum += 1.0 / (s - x[m]);
    return lagrange_at(x, n, a, s) * sum;
}

void derivative_matrix(const double *x, int n, double D[6][6]) {
    double bw[6];
    for (int a = 0; a < n; ++a) {
        double prod = 1.0;
        for (int m = 0; m < n; ++m)
            if (m != a) prod *= (x[a] - x[m]);
        bw[a] = 1.0 / prod;
    }
    for (int i = 0; i < n; ++i) {
        double diag = 0.0;
        for (int a = 0; a < n; ++a) {
            if (a == i) continue;
            D[i][a] = (bw[a] / bw[i]) / (x[i] - x[a]);
            diag -= D[i][a];
        }
        D[i][i] = diag;
    }
}

template <typename Real>
RefData<Real> make_ref(int order) {
    const int n = order + 1;
    double x[6], w[6], D[6][6];
    gauss_rule(n, x, w);
    derivative_matrix(x, n, D);
    RefData<Real> r;
    std::memset(&r, 0, sizeof(r));
    for (int a = 0; a < n; ++a) {
        const double lm = lagrange_at(x, n, a, -1.0), lp = lagrange_at(x, n, a, 1.0);
        r.lm[a] = (Real)lm;
        r.lp[a] = (Real)lp;
        r.liftm[a] = (Real)(lm / w[a]);
        r.liftp[a] = (Real)(lp / w[a]);
        r.xi[a] = (Real)x[a];
        r.w[a] = (Real)w[a];
        for (int i = 0; i < n; ++i) r.dhat[a][i] = (Real)(w[i] / w[a] * D[i][a]);
        for (int i = 0; i < n; ++i) r.dmat[i][a] = (Real)D[i][a];
        const double dlm = lagrange_deriv_at(x, n, a, -1.0), dlp = lagrange_deriv_at(x, n, a, 1.0);
        r.dlm[a] = (Real)dlm;
        r.dlp[a] = (Real)dlp;
        r.dliftm[a] = (Real)(dlm / w[a]);
        r.dliftp[a] = (Real)(dlp / w[a]);
    }
    return r;
}

// ---- hydrostatic column of the warm-bubble workload ------------------------
struct ColumnState {
    double rho_d, rho_v, rho_m, T, E, p;
};

double rho_vs_host(double T) {
    const double es = kEref * std::pow(T / kTref, kEsA) * std::exp(kEsB * (1.0 / kTref - 1.0 / T));
    return es / (kRv * T);
}

// p = (rho_d R_d + rho_v R_v) T, rho_v = min(rho_vs(T), qt rho_d): closed form per branch
ColumnState moist_at(double p, double T, double qt) {
    ColumnState c;
    const double rvs = rho_vs_host(T);
    double rd = p / (T * (kRd + qt * kRv));
    double rv = qt * rd;
    if (qt * rd > rvs) {
        rd = (p - rvs * kRv * T) / (kRd * T);
        rv = rvs;
    }
    c.rho_d = rd;
    c.rho_v = rv;
    c.p = p;
    c.rho_m = qt * rd;
    c.T = T;
    c.E = (kCvd * rd + kCvv * rv + kCl * (c.rho_m - rv)) * (T - kTref) + rv * kLprime;
    return c;
}

// Classical RK4 for dp/dz = -(rho_d + rho_m) g, T = theta (p/p_ref)^(R_d/c_pd),
// qt = qt0 (1 - z/H); steps <= 1 m landing on every requested level.
void column(const std::vector<double> &z, double theta, double p_s, double qt0, double H, double g,
            std::vector<ColumnState> &out) {
    const double kappa = kRd / kCpd;
    std::vector<size_t> order(z.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return z[a] < z[b]; });
    auto rhs = [&](double zz, double p) {
        const double T = theta * std::pow(p / kPref, kappa);
        const ColumnState c = moist_at(p, T, qt0 * (1.0 - zz / H));
        return -(c.rho_d + c.rho_m) * g;
    };
    out.assign(z.size(), ColumnState());
    double zc = 0.0, p = p_s;
    for (size_t idx : order) {
        const double zt = z[idx];
        if (zt > zc) {
            const int n = (int)std::ceil((zt - zc) / 1.0);
            const double hs = (zt - zc) / n;
            for (int i = 0; i < n; ++i) {
                const double k1 = rhs(zc, p);
                const double k2 = rhs(zc + 0.5 * hs, p + 0.5 * hs * k1);
                const double k3 = rhs(zc + 0.5 * hs, p + 0.5 * hs * k2);
                const double k4 = rhs(zc + hs, p + hs * k3);
                p += hs * (k1 + 2.0 * k2 + 2.0 * k3 + k4) / 6.0;
                zc += hs;
            }
            zc = zt;
        }
        const double T = theta * std::pow(p / kPref, kappa);
        out[idx] = moist_at(p, T, qt0 * (1.0 - zt / H));   // at rest: E is internal energy
    }
}

}  // namespace

namespace dgm {
// The float64 reference tables of order k with the volume derivative and
// lift coefficients scaled by 2/h_j of a mesh: the tables every float64 stage
// kernel takes (dg_init_mesh, dg_rhs_noalloc).
RefData<double> scaled_ref64(int order, const double two_over_h[3]) {
    RefData<double> r = make_ref<double>(order);
    for (int j = 0; j < 3; ++j)
        for (int a = 0; a < 6; ++a) {
            for (int i = 0; i < 6; ++i) r.dhat_s[j][a][i] = two_over_h[j] * r.dhat[a][i];
            const double sc = two_over_h[j];
            r.liftm_s[j][a] = sc * r.liftm[a];
            r.liftp_s[j][a] = sc * r.liftp[a];
            r.dliftm_s[j][a] = sc * sc * r.dliftm[a];
            r.dliftp_s[j][a] = sc * sc * r.dliftp[a];
        }
    return r;
}
}  // namespace dgm

#include "dg_ctx.h"

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? DG_OK : DG_ECUDA; }

template <typename Real>
KArgs<Real> base_args(const dg_ctx *c, const RefData<Real> &ref) {
    KArgs<Real> A;
    std::memset(&A, 0, sizeof(A));
    A.M = c->M;
    A.ref = ref;
    A.derived = (Real *)c->derived;
    A.bnode = (const Real *)c->bnode_r;
    A.bface = (const Real *)c->bface_r;
    A.bnode_d = c->bnode_d;
    A.rvs_tab = c->rvs_tab;
    A.bsplit = c->bsplit;
    A.fbuf = (Real *)c->fbuf;
    A.ftab = c->ftab;
    A.alphaK = (Real *)c->alphaK;
    A.alphaV = (const Real *)c->alphaV;
    A.flags = c->flags;
    A.fallout = c->fallout;
    return A;
}

// Host transfers in kChunks chunks of whole element tiles (the stage and
// prepare tiles), on the context's second stream up_stream
constexpr int kChunks = 8;

int ensure_up_stream(dg_ctx *c) {
    if (c->up_stream) return DG_OK;
    if (cudaStreamCreateWithFlags(&c->up_stream, cudaStreamNonBlocking) != cudaSuccess) return DG_ECUDA;
    for (cudaEvent_t &e : c->up_ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return DG_ECUDA;
    return DG_OK;
}

// element tiles [t0, t1) of chunk k
void chunk_tiles(const dg_ctx *c, int k, long long &t0, long long &t1) {
    const long long tiles = (c->ne + c->epb - 1) / c->epb;
    t0 = tiles * k / kChunks;
    t1 = tiles * (k + 1) / kChunks;
}

// the state values of chunk k's elements, one copy per field, on up_stream
int copy_chunk(dg_ctx *c, int k, void *dst, const void *src, cudaMemcpyKind kind) {
    long long t0, t1;
    chunk_tiles(c, k, t0, t1);
    const long long e0 = std::min(c->ne, t0 * c->epb), e1 = std::min(c->ne, t1 * c->epb);
    const size_t fstride = (size_t)c->nodes * c->rsz;   // bytes of one field
    const size_t ebytes = (size_t)c->np * c->rsz;       // bytes of one element in a field
    for (int f = 0; f < c->nf && e1 > e0; ++f) {
        const size_t off = (size_t)f * fstride + (size_t)e0 * ebytes;
        if (cudaMemcpyAsync((char *)dst + off, (const char *)src + off, (size_t)(e1 - e0) * ebytes, kind,
                            c->up_stream) != cudaSuccess)
            return DG_ECUDA;
    }
    return DG_OK;
}

// split and traces of state U into trace buffer tb; ntiles > 0: only the
// element tiles [tile0, tile0 + ntiles)
template <typename Real>
int do_prepare(dg_ctx *c, const Launchers<Real> *L, const RefData<Real> &ref, const void *U, int tb,
               int tile0, int ntiles) {
    KArgs<Real> A = base_args<Real>(c, ref);
    A.Uin = (const Real *)U;
    A.trace_out = (Real *)c->trace[tb];
    A.dtrace_out = (Real *)c->dtrace[tb];
    A.tile0 = tile0;
    A.ntiles = ntiles;
    return cuda_status(L->prepare(A, c->diff, c->stream));
}

int prepare(dg_ctx *c, const void *U, int tb, int tile0 = 0, int ntiles = 0) {
    return c->fp32 ? do_prepare<float>(c, c->L32, c->ref32, U, tb, tile0, ntiles)
                   : do_prepare<double>(c, c->L64, c->ref64, U, tb, tile0, ntiles);
}

// Upload of a host state in kChunks chunks of whole element tiles: the
// copies of chunk i (one per field) run on up_stream while the stream
// splits chunk i - 1 (k_prepare over its tiles), so the split of an
// uploaded state hides behind the copy.  Leaves the split and the traces
// of the new state in trace buffer 0, as dg_step's own prepare would.
int upload_and_prepare(dg_ctx *c, const void *host) {
    if (ensure_up_stream(c) != DG_OK) return DG_ECUDA;
    // nothing on the stream may still read U[0] when the copies overwrite it
    if (cudaEventRecord(c->up_ev[kChunks], c->stream) != cudaSuccess ||
        cudaStreamWaitEvent(c->up_stream, c->up_ev[kChunks], 0) != cudaSuccess)
        return DG_ECUDA;
    for (int k = 0; k < kChunks; ++k) {
        long long t0, t1;
        chunk_tiles(c, k, t0, t1);
        if (copy_chunk(c, k, c->U[0], host, cudaMemcpyHostToDevice) != DG_OK) return DG_ECUDA;
        if (cudaEventRecord(c->up_ev[k], c->up_stream) != cudaSuccess ||
            cudaStreamWaitEvent(c->stream, c->up_ev[k], 0) != cudaSuccess)
            return DG_ECUDA;
        if (t1 > t0) {
            const int st = prepare(c, c->U[0], 0, (int)t0, (int)(t1 - t0));
            if (st != DG_OK) return st;
        }
    }
    c->parity = 0;
    c->derived_valid = true;
    return DG_OK;
}

// last: the stage that ends a time step (the sponge layer acts there);
// fall_w: the stage's weight b_s dt in the step for the rain fall-out (0: the
// stage adds nothing to it)
// chunk_ev: launch the stage kernel in kChunks chunks of element tiles and
// record chunk_ev[k] after chunk k (a download can follow chunk by chunk);
// null: one launch
template <typename Real>
int do_stage(dg_ctx *c, const Launchers<Real> *L, const RefData<Real> &ref, int mode, const void *Uin,
             const void *Un, void *Uout, int tin, double alpha, double beta, double gdt, bool last,
             double fall_w, cudaEvent_t *chunk_ev) {
    KArgs<Real> A = base_args<Real>(c, ref);
    A.fall_w = fall_w;
    if (fall_w == 0.0 || mode != MODE_STAGE) A.fallout = nullptr;
    A.Uin = (const Real *)Uin;
    A.Un = (const Real *)Un;
    A.Uout = (Real *)Uout;
    A.trace_in = (const Real *)c->trace[tin];
    A.trace_out = (Real *)c->trace[1 - tin];
    A.dtrace_in = (const Real *)c->dtrace[tin];
    A.dtrace_out = (Real *)c->dtrace[1 - tin];
    A.alpha = (Real)alpha;
    A.beta = (Real)beta;
    A.gdt = (Real)gdt;
    A.sponge = (last && mode == MODE_STAGE) ? (const Real *)c->sponge : nullptr;
    if (c->diff) {
        const int st = cuda_status(L->alpha_vertex(A, c->stream));
        if (st != DG_OK) return st;
    }
    if (c->column) return cuda_status(L->column(A, mode, c->stream));
    if (c->face_pass) {
        const int st = cuda_status(L->face(A, c->diff, c->stream));
        if (st != DG_OK) return st;
    }
    if (!chunk_ev) return cuda_status(L->stage(A, mode, c->face_pass, c->diff, c->stream));
    for (int k = 0; k < kChunks; ++k) {
        long long t0, t1;
        chunk_tiles(c, k, t0, t1);
        if (t1 > t0) {
            A.tile0 = (int)t0;
            A.ntiles = (int)(t1 - t0);
            const int st = cuda_status(L->stage(A, mode, c->face_pass, c->diff, c->stream));
            if (st != DG_OK) return st;
        }
        if (cudaEventRecord(chunk_ev[k], c->stream) != cudaSuccess) return DG_ECUDA;
    }
    return DG_OK;
}

int stage(dg_ctx *c, int mode, const void *Uin, const void *Un, void *Uout, int tin, double alpha,
          double beta, double gdt, bool last = false, double fall_w = 0.0,
          cudaEvent_t *chunk_ev = nullptr) {
    return c->fp32 ? do_stage<float>(c, c->L32, c->ref32, mode, Uin, Un, Uout, tin, alpha, beta, gdt,
                                     last, fall_w, chunk_ev)
                   : do_stage<double>(c, c->L64, c->ref64, mode, Uin, Un, Uout, tin, alpha, beta, gdt,
                                      last, fall_w, chunk_ev);
}

// the fall-out starts again from zero with every new state
int reset_fallout(dg_ctx *c) {
    if (!c->fallout) return DG_OK;
    return cudaMemsetAsync(c->fallout, 0, sizeof(double) * c->fallout_len, c->stream) == cudaSuccess
               ? DG_OK
               : DG_ECUDA;
}

void release(dg_ctx *c) {
    void *ptrs[] = {c->U[0], c->U[1], c->derived, c->trace[0], c->trace[1], c->bnode_d,
                    c->bface_d, c->bnode_r, c->bface_r, c->flags, c->partials, c->rvs_tab,
                    c->adjX[0], c->adjX[1], c->adjX[2], c->adjL[0], c->adjL[1], c->adjL[2],
                    c->ubar_part, c->tadj, c->bsplit, c->fbuf, c->ftab, c->alphaK, c->alphaV,
                    c->dtrace[0], c->dtrace[1], c->sponge, c->fallout};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

// float32 copies of the mesh constants (used by the float32 forms)
void mesh_float_copies(MeshData &M) {
    for (int j = 0; j < 3; ++j) {
        M.two_over_h_f[j] = (float)M.two_over_h[j];
        M.sigma_pen_f[j] = (float)M.sigma_pen[j];
    }
    M.g_f = (float)M.g;
    M.kvr_f = (float)M.kvr;
    M.rho_w_f = (float)M.rho_w;
    M.jac_f = (float)M.jac;
    M.alpha_pre_f = (float)M.alpha_pre;
}

// face grid of the face pass; returns the length (in elements) of its
// face-major buffer [faces normal to e_0 | e_1 | e_2][per_point][NFP1]
long long set_face_layout(dg_ctx *c, int per_point) {
    MeshData &M = c->M;
    const dg_config &g = c->cfg;
    for (int j = 0; j < 3; ++j) {
        M.nfn[j] = (j < g.dim) ? M.n[j] + (M.periodic[j] ? 0 : 1) : 1;
        M.nv[j] = M.nfn[j];
        long long nfj = 0;
        if (j < g.dim) {
            nfj = 1;
            for (int i = 0; i < g.dim; ++i) nfj *= (i == j) ? M.nfn[i] : M.n[i];
        }
        M.nfaces[j] = (int)nfj;
        M.fblk[j] = (int)((nfj * c->nfp1 + kFaceThreads - 1) / kFaceThreads);
    }
    return ((long long)M.nfaces[0] + M.nfaces[1] + M.nfaces[2]) * per_point * c->nfp1;
}

// index in the face-major face buffer of every element's 2D faces, [ne][2D]
// (face 2j + s: the low (s = 0) or high (s = 1) face normal to e_j; the high
// face of the last element of a periodic row is the row's face 0)
std::vector<int> face_table(const dg_ctx *c) {
    const MeshData &M = c->M;
    const int d = c->cfg.dim;
    std::vector<int> tab((size_t)c->ne * 2 * d);
    for (long long e = 0; e < c->ne; ++e) {
        const int im[3] = {(int)(e % M.n[0]), (int)((e / M.n[0]) % M.n[1]),
                           d == 3 ? (int)(e / ((long long)M.n[0] * M.n[1])) : 0};
        long long off = 0;
        for (int j = 0; j < d; ++j) {
            for (int side = 0; side < 2; ++side) {
                int f[3] = {im[0], im[1], im[2]};
                f[j] += side;
                if (f[j] == M.n[j] && M.periodic[j]) f[j] = 0;
                const long long n0 = j == 0 ? M.nfn[0] : M.n[0], n1 = j == 1 ? M.nfn[1] : M.n[1];
                tab[(size_t)e * 2 * d + 2 * j + side] = (int)(off + f[0] + n0 * (f[1] + n1 * f[2]));
            }
            off += M.nfaces[j];
        }
    }
    return tab;
}

int alloc(dg_ctx *c, void **p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return DG_ENOMEM;
    }
    c->device_bytes += bytes;
    return DG_OK;
}

int upload_base(dg_ctx *c, const double *node_tab, const double *face_tab) {
    const int nn = c->M.nzlev_node, nfz = c->M.nzlev_face;
    cudaError_t e = cudaMemcpyAsync(c->bnode_d, node_tab, sizeof(double) * 4 * nn,
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->bface_d, face_tab, sizeof(double) * 4 * nfz, cudaMemcpyHostToDevice,
                            c->stream);
    if (e != cudaSuccess) return DG_ECUDA;
    if (c->fp32) {
        std::vector<float> fn(4 * nn), ff(4 * nfz);
        for (int i = 0; i < 4 * nn; ++i) fn[i] = (float)node_tab[i];
        for (int i = 0; i < 4 * nfz; ++i) ff[i] = (float)face_tab[i];
        e = cudaMemcpyAsync(c->bnode_r, fn.data(), sizeof(float) * fn.size(), cudaMemcpyHostToDevice,
                            c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->bface_r, ff.data(), sizeof(float) * ff.size(),
                                cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // host vectors go out of scope
        if (e != cudaSuccess) return DG_ECUDA;
    } else {
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return DG_ECUDA;
    }
    if (c->bsplit) {
        // the split of the base state, per node level, for the perturbation-form split
        k_base_split<<<(nn + 127) / 128, 128, 0, c->stream>>>(c->bnode_d, nn, c->bsplit, c->rvs_tab);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess)
            return DG_ECUDA;
    }
    c->base_set = true;
    c->derived_valid = false;
    return DG_OK;
}

int ensure_adjoint(dg_ctx *c) {
    if (c->ubar_part) return DG_OK;
    const size_t state = (size_t)c->nodes * c->nf * sizeof(double);
    const size_t trace = (size_t)2 * c->cfg.dim * c->ntr * c->ne * c->nfp1 * sizeof(double);
    int st = DG_OK;
    for (int i = 0; i < 3 && st == DG_OK; ++i) st = alloc(c, &c->adjX[i], state);
    for (int i = 0; i < 3 && st == DG_OK; ++i) st = alloc(c, (void **)&c->adjL[i], state);
    if (st == DG_OK) st = alloc(c, (void **)&c->tadj, trace);
    if (st == DG_OK) st = alloc(c, (void **)&c->ubar_part, (size_t)c->nodes * c->ntr * sizeof(double));
    return st;
}

AdjArgs adj_args(const dg_ctx *c, const void *U, const double *w, double *out, double alpha,
                 double beta, double gamma) {
    AdjArgs A;
    std::memset(&A, 0, sizeof(A));
    A.M = c->M;
    A.ref = c->ref64;
    A.U = (const double *)U;
    A.derived = (const double *)c->derived;
    A.trace = (const double *)c->trace[0];
    A.bnode = c->bnode_d;
    A.bface = c->bface_d;
    A.rvs_tab = c->rvs_tab;
    A.w = w;
    A.ubar_part = c->ubar_part;
    A.tadj = c->tadj;
    A.out = out;
    A.alpha = alpha;
    A.beta = beta;
    A.gamma = gamma;
    return A;
}

// out = alpha out + beta w + gamma (dR/dU (U))^T w
int rhs_adjoint_into(dg_ctx *c, const void *U, const double *w, double *out, double alpha,
                     double beta, double gamma) {
    c->derived_valid = false;
    int st = prepare(c, U, 0);
    if (st != DG_OK) return st;
    AdjArgs A = adj_args(c, U, w, out, alpha, beta, gamma);
    if (c->LA->local(A, c->stream) != cudaSuccess) return DG_ECUDA;
    if (c->LA->gather(A, c->stream) != cudaSuccess) return DG_ECUDA;
    return DG_OK;
}

}  // namespace

int dgm::ctx_prepare(dg_ctx *c, const void *U, int tb) { return prepare(c, U, tb); }

// ---------------------------------------------------------------------------
extern "C" {

const char *dg_strerror(int code) {
    switch (code) {
        case DG_OK: return "ok";
        case DG_EINVAL: return "invalid argument or size";
        case DG_ENOMEM: return "device allocation failed";
        case DG_ECUDA: return "CUDA error";
        case DG_ENOCONV: return "Newton split did not converge at some node";
        case DG_ENONPHYS: return "non-physical or non-finite state";
        case DG_ESTATE: return "base state or state not set";
        case DG_ENOTIMPL: return "not implemented for this configuration";
        default: return "unknown status";
    }
}

int dg_gauss_legendre(int n, double *x, double *w) {
    if (n < 1 || n > 6 || !x || !w) return DG_EINVAL;
    gauss_rule(n, x, w);
    return DG_OK;
}

int dg_init_mesh(dg_ctx **out, const dg_config *cfg, void *cuda_stream) {
    if (!out || !cfg) return DG_EINVAL;
    *out = nullptr;
    const dg_config &g = *cfg;
    if (g.dim != 2 && g.dim != 3) return DG_EINVAL;
    if (g.order < 1 || g.order > 5) return DG_EINVAL;
    if (g.precision != DG_FP64 && g.precision != DG_FP32_BULK && g.precision != DG_FP32_PERT &&
        g.precision != DG_FP64_FFC)
        return DG_EINVAL;
    if (g.rain != 0 && g.rain != 1) return DG_EINVAL;
    if (g.faces != DG_FACES_AUTO && g.faces != DG_FACES_INLINE && g.faces != DG_FACES_PASS &&
        g.faces != DG_FACES_COLUMN)
        return DG_EINVAL;
    long long ne = 1;
    for (int j = 0; j < g.dim; ++j) {
        if (g.n[j] < 1 || !(g.L[j] > 0.0) || !std::isfinite(g.L[j])) return DG_EINVAL;
        ne *= g.n[j];
    }
    if (!std::isfinite(g.g)) return DG_EINVAL;
    const int p1 = g.order + 1;
    const int np = g.dim == 2 ? p1 * p1 : p1 * p1 * p1;
    const int nf = (g.rain ? 4 : 3) + g.dim;
    if (ne * np * (long long)(nf + 3) * 2 > 2147483647LL) return DG_EINVAL;
    if (g.faces == DG_FACES_COLUMN && (g.precision == DG_FP64 || g.precision == DG_FP64_FFC))
        return DG_ENOTIMPL;

    dg_ctx *c = new (std::nothrow) dg_ctx();
    if (!c) return DG_ENOMEM;
    c->cfg = g;
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return DG_ECUDA;
    }
    c->fp32 = (g.precision == DG_FP32_BULK || g.precision == DG_FP32_PERT);
    c->rsz = c->fp32 ? sizeof(float) : sizeof(double);
    if (c->fp32) {
        c->L32 = g.dim == 2 ? launchers_d2_f32(g.order, g.rain) : launchers_d3_f32(g.order, g.rain);
        c->nf = c->L32->nf; c->np = c->L32->np; c->nfp1 = c->L32->nfp1;
        c->nd = c->L32->nd; c->ntr = c->L32->ntr; c->epb = c->L32->epb;
    } else {
        if (g.precision == DG_FP64_FFC)
            c->L64 = g.dim == 2 ? launchers_d2_f64ff(g.order, g.rain) : launchers_d3_f64ff(g.order, g.rain);
        else
            c->L64 = g.dim == 2 ? launchers_d2_f64(g.order, g.rain) : launchers_d3_f64(g.order, g.rain);
        c->LA = g.dim == 2 ? adj_launchers_d2(g.order, g.rain) : adj_launchers_d3(g.order, g.rain);
        c->nf = c->L64->nf; c->np = c->L64->np; c->nfp1 = c->L64->nfp1;
        c->nd = c->L64->nd; c->ntr = c->L64->ntr; c->epb = c->L64->epb;
    }
    c->ne = ne;
    c->nodes = ne * np;

    MeshData &M = c->M;
    std::memset(&M, 0, sizeof(M));
    for (int j = 0; j < 3; ++j) {
        M.n[j] = j < g.dim ? g.n[j] : 1;
        M.h[j] = j < g.dim ? g.L[j] / g.n[j] : 1.0;
        M.two_over_h[j] = 2.0 / M.h[j];
        M.periodic[j] = (j < g.dim - 1) ? ((g.periodic_mask >> j) & 1) : 0;
    }
    M.ne = (int)ne;
    const int nvert = g.n[g.dim - 1];
    M.nzlev_node = nvert * p1;
    M.nzlev_face = nvert + 1;
    M.g = g.g;
    M.rho_w = g.rho_w;
    // v0 Gamma(4.5)/6 (pi N0)^(-1/8) with N0 = 8e6 m^-4, v0 = 130 m^(1/2)/s (Section 2.1)
    M.kvr = 130.0 * std::tgamma(4.5) / 6.0 * std::pow(M_PI * 8.0e6, -0.125);
    M.jac = 1.0;
    for (int j = 0; j < g.dim; ++j) M.jac *= M.h[j] / 2.0;
    M.rain_floor = kRainFloorLin;
    M.rain_d8 = 0.125 * std::pow(kRainFloorLin, -0.875);
    M.rain_d16 = 0.0625 * std::pow(kRainFloorLin, -0.9375);
    M.pert_split = (g.precision == DG_FP32_PERT) ? 1 : 0;
    M.newton_cap = kMaxNewton;
    // face grid and the face-pass flux buffer layout
    // the face pass is the faster schedule for every precision on GB300
    // (measured: float64 -21 %, float32 forms -8 to -11 % per step)
    c->face_pass = g.faces == DG_FACES_AUTO || g.faces == DG_FACES_PASS;
    c->column = g.faces == DG_FACES_COLUMN;
    const long long fbuf_len = set_face_layout(c, nf);
    mesh_float_copies(M);
    // the volume derivative and lift tables pre-scaled by 2/h_j of this
    // mesh, float64 and their float32 roundings
    c->ref64 = scaled_ref64(g.order, M.two_over_h);
    c->ref32 = make_ref<float>(g.order);
    for (int j = 0; j < 3; ++j)
        for (int a = 0; a < 6; ++a) {
            for (int i = 0; i < 6; ++i) c->ref32.dhat_s[j][a][i] = (float)c->ref64.dhat_s[j][a][i];
            c->ref32.liftm_s[j][a] = (float)c->ref64.liftm_s[j][a];
            c->ref32.liftp_s[j][a] = (float)c->ref64.liftp_s[j][a];
            c->ref32.dliftm_s[j][a] = (float)c->ref64.dliftm_s[j][a];
            c->ref32.dliftp_s[j][a] = (float)c->ref64.dliftp_s[j][a];
        }

    // z-levels
    c->z_node.resize(M.nzlev_node);
    c->z_face.resize(M.nzlev_face);
    const double hz = M.h[g.dim - 1];
    for (int iz = 0; iz < nvert; ++iz)
        for (int a = 0; a < p1; ++a)
            c->z_node[iz * p1 + a] = iz * hz + (1.0 + (double)c->ref64.xi[a]) * hz * 0.5;
    for (int iz = 0; iz <= nvert; ++iz) c->z_face[iz] = iz * hz;

    DeviceGuard dg(c->device);
    const size_t state = (size_t)c->nodes * nf * c->rsz;
    const size_t trace = (size_t)2 * g.dim * c->ntr * ne * c->nfp1 * c->rsz;
    c->nred = std::min<long long>(kGridStrideBlocks, (c->nodes + kRedThreads - 1) / kRedThreads);
    int st = DG_OK;
    if (st == DG_OK) st = alloc(c, &c->U[0], state);
    if (st == DG_OK) st = alloc(c, &c->U[1], state);
    if (st == DG_OK) st = alloc(c, &c->derived, (size_t)c->nodes * c->nd * c->rsz);
    if (st == DG_OK) st = alloc(c, &c->trace[0], trace);
    if (st == DG_OK) st = alloc(c, &c->trace[1], trace);
    if (st == DG_OK) st = alloc(c, (void **)&c->bnode_d, sizeof(double) * 4 * M.nzlev_node);
    if (st == DG_OK) st = alloc(c, (void **)&c->bface_d, sizeof(double) * 4 * M.nzlev_face);
    if (c->fp32) {
        if (st == DG_OK) st = alloc(c, &c->bnode_r, sizeof(float) * 4 * M.nzlev_node);
        if (st == DG_OK) st = alloc(c, &c->bface_r, sizeof(float) * 4 * M.nzlev_face);
    } else {
        c->bnode_r = nullptr;
        c->bface_r = nullptr;
    }
    if (st == DG_OK) st = alloc(c, (void **)&c->flags, sizeof(unsigned long long) * 2);
    if (st == DG_OK) st = alloc(c, (void **)&c->partials, sizeof(double) * kNRed * c->nred);
    if (st == DG_OK) st = alloc(c, (void **)&c->rvs_tab, sizeof(double) * kTabStride * kTabN);
    if (st == DG_OK && M.pert_split)
        st = alloc(c, (void **)&c->bsplit, sizeof(float) * kBsN * M.nzlev_node);
    if (st == DG_OK && c->face_pass) st = alloc(c, &c->fbuf, (size_t)fbuf_len * c->rsz);
    if (st == DG_OK && c->face_pass) {
        const std::vector<int> tab = face_table(c);
        st = alloc(c, (void **)&c->ftab, sizeof(int) * tab.size());
        if (st == DG_OK && cudaMemcpy(c->ftab, tab.data(), sizeof(int) * tab.size(),
                                      cudaMemcpyHostToDevice) != cudaSuccess)
            st = DG_ECUDA;
    }
    if (st == DG_OK && g.rain) {
        // fall-out accumulator: the points of the bottom and top wall faces
        c->fallout_len = (size_t)2 * (ne / g.n[g.dim - 1]) * c->nfp1;
        st = alloc(c, (void **)&c->fallout, sizeof(double) * c->fallout_len);
        if (st == DG_OK) st = reset_fallout(c);
    }
    if (st == DG_OK && cudaMemsetAsync(c->flags, 0, 2 * sizeof(unsigned long long), c->stream) != cudaSuccess)
        st = DG_ECUDA;
    if (st == DG_OK) {
        k_fill_rvs_table<<<(kTabN + 255) / 256, 256, 0, c->stream>>>(c->rvs_tab);
        if (cudaGetLastError() != cudaSuccess) st = DG_ECUDA;
    }
    if (st != DG_OK) {
        release(c);
        delete c;
        return st;
    }
    if (!c->fp32) {
        // the float64 tables serve both the split and the flux arithmetic
        c->bnode_r = c->bnode_d;
        c->bface_r = c->bface_d;
    }
    *out = c;
    return DG_OK;
}

void dg_free(dg_ctx *c) {
    if (!c) return;
    {
        DeviceGuard dg(c->device);
        cudaStreamSynchronize(c->stream);
        if (c->up_stream) {
            cudaStreamSynchronize(c->up_stream);
            cudaStreamDestroy(c->up_stream);
            for (cudaEvent_t e : c->up_ev)
                if (e) cudaEventDestroy(e);
        }
        if (c->fp32) {
            release(c);
        } else {
            c->bnode_r = nullptr;
            c->bface_r = nullptr;
            release(c);
        }
    }
    delete c;
}

int dg_get_info(const dg_ctx *c, dg_info *info) {
    if (!c || !info) return DG_EINVAL;
    info->n_fields = c->nf;
    info->nodes_per_elem = c->np;
    info->face_points_per_face = c->nfp1;
    info->n_zlev_node = c->M.nzlev_node;
    info->n_zlev_face = c->M.nzlev_face;
    info->elems_per_block = c->epb;
    info->n_elem = c->ne;
    info->n_nodes = c->nodes;
    info->n_dofs = c->nodes * c->nf;
    info->state_bytes = (size_t)c->nodes * c->nf * c->rsz;
    info->device_bytes = c->device_bytes;
    info->launches_per_stage = c->face_pass ? 2 : 1;   // column march and inline faces: 1
    return DG_OK;
}

int dg_zlevels(const dg_ctx *c, double *z_node, double *z_face) {
    if (!c || !z_node || !z_face) return DG_EINVAL;
    std::copy(c->z_node.begin(), c->z_node.end(), z_node);
    std::copy(c->z_face.begin(), c->z_face.end(), z_face);
    return DG_OK;
}

int dg_set_base_state(dg_ctx *c, const double *node_tab, const double *face_tab) {
    if (!c || !node_tab || !face_tab) return DG_EINVAL;
    DeviceGuard dg(c->device);
    return upload_base(c, node_tab, face_tab);
}

int dg_init_bubble(dg_ctx *c, const dg_bubble *b, const double *noise, int where) {
    if (!c || !b) return DG_EINVAL;
    if (where != DG_HOST && where != DG_DEVICE) return DG_EINVAL;
    if (!(b->H > 0.0) || !(b->p_s > 0.0) || !(b->theta > 0.0)) return DG_EINVAL;
    for (int j = 0; j < c->cfg.dim; ++j)
        if (!(b->radius[j] > 0.0)) return DG_EINVAL;
    DeviceGuard dg(c->device);
    const int nn = c->M.nzlev_node, nfz = c->M.nzlev_face;
    std::vector<double> z(c->z_node);
    z.insert(z.end(), c->z_face.begin(), c->z_face.end());
    std::vector<ColumnState> col;
    column(z, b->theta, b->p_s, b->qt0, b->H, c->cfg.g, col);
    std::vector<double> tn(4 * nn), tf(4 * nfz);
    for (int i = 0; i < nn + nfz; ++i) {
        const ColumnState &s = col[i];
        const double p = s.p;
        double *tab = i < nn ? tn.data() : tf.data();
        const int k = i < nn ? i : i - nn, n = i < nn ? nn : nfz;
        tab[k] = s.rho_d;
        tab[n + k] = s.rho_m;
        tab[2 * n + k] = s.E;
        tab[3 * n + k] = p;
    }
    int st = upload_base(c, tn.data(), tf.data());
    if (st != DG_OK) return st;
    BubbleArgs B;
    B.theta = b->theta;
    B.qt0 = b->qt0;
    B.H = b->H;
    B.amplitude = b->amplitude;
    for (int j = 0; j < 3; ++j) {
        B.centre[j] = b->centre[j];
        B.radius[j] = j < c->cfg.dim ? b->radius[j] : 1.0;
    }
    B.noise = nullptr;
    if (noise) {
        if (where == DG_DEVICE) {
            B.noise = noise;
        } else {
            // stage the host noise in the derived-field buffer (stale here, >= 8 B per node)
            if (cudaMemcpyAsync(c->derived, noise, sizeof(double) * c->nodes, cudaMemcpyHostToDevice,
                                c->stream) != cudaSuccess)
                return DG_ECUDA;
            B.noise = (const double *)c->derived;
        }
    }
    cudaError_t e;
    if (c->fp32) {
        KArgs<float> A = base_args<float>(c, c->ref32);
        A.Uout = (float *)c->U[0];
        e = c->L32->init_bubble(A, B, c->stream);
    } else {
        KArgs<double> A = base_args<double>(c, c->ref64);
        A.Uout = (double *)c->U[0];
        e = c->L64->init_bubble(A, B, c->stream);
    }
    if (e != cudaSuccess) return DG_ECUDA;
    if (reset_fallout(c) != DG_OK) return DG_ECUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return DG_ECUDA;
    c->state_set = true;
    c->derived_valid = false;
    return DG_OK;
}

int dg_set_state(dg_ctx *c, const void *U, int where) {
    if (!c || !U || (where != DG_HOST && where != DG_DEVICE)) return DG_EINVAL;
    DeviceGuard dg(c->device);
    c->derived_valid = false;
    if (reset_fallout(c) != DG_OK) return DG_ECUDA;
    if (where == DG_HOST && c->base_set) {
        // the split of the new state overlaps its upload
        const int st = upload_and_prepare(c, U);
        if (st != DG_OK) {
            c->derived_valid = false;
            return st;
        }
        c->state_set = true;
        return DG_OK;
    }
    const size_t bytes = (size_t)c->nodes * c->nf * c->rsz;
    cudaError_t e = cudaMemcpyAsync(c->U[0], U, bytes,
                                    where == DG_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                    c->stream);
    if (e != cudaSuccess) return DG_ECUDA;
    c->state_set = true;
    return DG_OK;
}

int dg_get_state(dg_ctx *c, void *U, int where) {
    if (!c || !U || (where != DG_HOST && where != DG_DEVICE)) return DG_EINVAL;
    if (!c->state_set) return DG_ESTATE;
    DeviceGuard dg(c->device);
    const size_t bytes = (size_t)c->nodes * c->nf * c->rsz;
    cudaError_t e = cudaMemcpyAsync(U, c->U[0], bytes,
                                    where == DG_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                    c->stream);
    if (e != cudaSuccess) return DG_ECUDA;
    if (where == DG_HOST && cudaStreamSynchronize(c->stream) != cudaSuccess) return DG_ECUDA;
    return DG_OK;
}

int dg_check_status(dg_ctx *c, long long counts[2]) {
    if (!c) return DG_EINVAL;
    DeviceGuard dg(c->device);
    unsigned long long h[2] = {0, 0};
    if (cudaMemcpyAsync(h, c->flags, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return DG_ECUDA;
    if (cudaMemsetAsync(c->flags, 0, sizeof(h), c->stream) != cudaSuccess) return DG_ECUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return DG_ECUDA;
    if (counts) {
        counts[0] = (long long)h[0];
        counts[1] = (long long)h[1];
    }
    if (h[1]) return DG_ENONPHYS;
    if (h[0]) return DG_ENOCONV;
    return DG_OK;
}

int dg_set_newton_limit(dg_ctx *c, int max_iterations) {
    if (!c || max_iterations < 1 || max_iterations > 1000) return DG_EINVAL;
    c->M.newton_cap = max_iterations;
    return DG_OK;
}

int dg_saturation_split(dg_ctx *c, const void *U, double *T, double *rho_v, double *rho_c,
                        double *p_prime, long long *n_unconverged) {
    if (!c || !U) return DG_EINVAL;
    if (!c->base_set) return DG_ESTATE;
    DeviceGuard dg(c->device);
    cudaError_t e;
    if (n_unconverged) {
        long long dummy[2];
        int st = dg_check_status(c, dummy);  // start from clean counters
        (void)st;
    }
    if (c->fp32) {
        KArgs<float> A = base_args<float>(c, c->ref32);
        A.Uin = (const float *)U;
        e = c->L32->split(A, T, rho_v, rho_c, p_prime, c->stream);
    } else {
        KArgs<double> A = base_args<double>(c, c->ref64);
        A.Uin = (const double *)U;
        e = c->L64->split(A, T, rho_v, rho_c, p_prime, c->stream);
    }
    if (e != cudaSuccess) return DG_ECUDA;
    if (n_unconverged) {
        long long cnt[2];
        int st = dg_check_status(c, cnt);
        *n_unconverged = cnt[0];
        if (st == DG_ENONPHYS) return st;
        if (st == DG_ECUDA) return st;
    }
    return DG_OK;
}

int dg_rhs(dg_ctx *c, const void *U, void *dUdt) {
    if (!c || !U || !dUdt || U == dUdt) return DG_EINVAL;
    if (!c->base_set) return DG_ESTATE;
    DeviceGuard dg(c->device);
    // the scratch derived fields and trace buffer 0 now describe U, not U^n
    c->derived_valid = false;
    int st = prepare(c, U, 0);
    if (st != DG_OK) return st;
    return stage(c, MODE_RHS, U, U, dUdt, 0, 0.0, 1.0, 1.0);
}

}  // extern "C"

namespace {

// nsteps SSPRK(4,3) steps on the context's stream; last_chunks: the final
// stage of the final step runs in chunks and records these events (for a
// download that follows it chunk by chunk)
int step_impl(dg_ctx *c, double dt, int nsteps, cudaEvent_t *last_chunks) {
    int st = DG_OK;
    if (!c->derived_valid) {
        st = prepare(c, c->U[0], 0);
        if (st != DG_OK) return st;
        c->parity = 0;
        c->derived_valid = true;
    }
    void *Un = c->U[0], *Uw = c->U[1];
    // SSPRK(4,3), Shu-Osher form (Remark 3.1):
    //   u1 = u + dt/2 L(u); u2 = u1 + dt/2 L(u1); u3 = 2/3 u + 1/3 u2 + dt/6 L(u2);
    //   u^{n+1} = u3 + dt/2 L(u3)
    for (int n = 0; n < nsteps && st == DG_OK; ++n) {
        // the fall-out weights are those of L(u_s) in u^{n+1} once the
        // stages are expanded: dt (1/6, 1/6, 1/6, 1/2)
        int p = c->parity;
        st = stage(c, MODE_STAGE, Un, Un, Uw, p, 0.0, 1.0, 0.5 * dt, false, dt / 6.0);
        p ^= 1;
        if (st == DG_OK) st = stage(c, MODE_STAGE, Uw, Uw, Uw, p, 0.0, 1.0, 0.5 * dt, false, dt / 6.0);
        p ^= 1;
        if (st == DG_OK)
            st = stage(c, MODE_STAGE, Uw, Un, Uw, p, 2.0 / 3.0, 1.0 / 3.0, dt / 6.0, false, dt / 6.0);
        p ^= 1;
        if (st == DG_OK)
            st = stage(c, MODE_STAGE, Uw, Uw, Un, p, 0.0, 1.0, 0.5 * dt, true, 0.5 * dt,
                       n + 1 == nsteps ? last_chunks : nullptr);
        p ^= 1;
        c->parity = p;
    }
    return st;
}

}  // namespace

extern "C" {

int dg_step_async(dg_ctx *c, double dt, int nsteps) {
    if (!c || nsteps < 0 || !std::isfinite(dt)) return DG_EINVAL;
    if (!c->base_set || !c->state_set) return DG_ESTATE;
    DeviceGuard dg(c->device);
    return step_impl(c, dt, nsteps, nullptr);
}

int dg_step_to_host(dg_ctx *c, double dt, int nsteps, void *U) {
    if (!c || !U || nsteps < 1 || !std::isfinite(dt)) return DG_EINVAL;
    if (!c->base_set || !c->state_set) return DG_ESTATE;
    DeviceGuard dg(c->device);
    if (ensure_up_stream(c) != DG_OK) return DG_ECUDA;
    // the column march is one launch per stage: no chunks, the download follows
    const bool chunked = !c->column;
    int st = step_impl(c, dt, nsteps, chunked ? c->up_ev : nullptr);
    if (st != DG_OK) return st;
    if (chunked) {
        for (int k = 0; k < kChunks; ++k) {
            if (cudaStreamWaitEvent(c->up_stream, c->up_ev[k], 0) != cudaSuccess) return DG_ECUDA;
            if (copy_chunk(c, k, U, c->U[0], cudaMemcpyDeviceToHost) != DG_OK) return DG_ECUDA;
        }
        // later work on the stream may overwrite U^n only after the download
        if (cudaEventRecord(c->up_ev[kChunks], c->up_stream) != cudaSuccess ||
            cudaStreamWaitEvent(c->stream, c->up_ev[kChunks], 0) != cudaSuccess ||
            cudaStreamSynchronize(c->up_stream) != cudaSuccess)
            return DG_ECUDA;
    } else if (cudaMemcpyAsync(U, c->U[0], (size_t)c->nodes * c->nf * c->rsz, cudaMemcpyDeviceToHost,
                               c->stream) != cudaSuccess) {
        return DG_ECUDA;
    }
    return dg_check_status(c, nullptr);
}

int dg_step(dg_ctx *c, double dt, int nsteps) {
    int st = dg_step_async(c, dt, nsteps);
    if (st != DG_OK) return st;
    return dg_check_status(c, nullptr);
}

int dg_reduce(dg_ctx *c, double out[DG_NREDUCE]) {
    if (!c || !out) return DG_EINVAL;
    if (!c->base_set || !c->state_set) return DG_ESTATE;
    DeviceGuard dg(c->device);
    if (!c->derived_valid) {
        int st = prepare(c, c->U[0], 0);
        if (st != DG_OK) return st;
        c->parity = 0;
        c->derived_valid = true;
    }
    cudaError_t e;
    if (c->fp32) {
        KArgs<float> A = base_args<float>(c, c->ref32);
        A.Uin = (const float *)c->U[0];
        e = c->L32->reduce(A, c->partials, c->nred, c->stream);
    } else {
        KArgs<double> A = base_args<double>(c, c->ref64);
        A.Uin = (const double *)c->U[0];
        e = c->L64->reduce(A, c->partials, c->nred, c->stream);
    }
    if (e != cudaSuccess) return DG_ECUDA;
    std::vector<double> h((size_t)kNRed * c->nred);
    if (cudaMemcpyAsync(h.data(), c->partials, sizeof(double) * h.size(), cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess)
        return DG_ECUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return DG_ECUDA;
    for (int r = 0; r < kNRed; ++r) out[r] = (r == 5 || r == 6) ? -INFINITY : 0.0;
    for (int b = 0; b < c->nred; ++b)
        for (int r = 0; r < kNRed; ++r) {
            const double v = h[(size_t)b * kNRed + r];
            out[r] = (r == 5 || r == 6) ? std::max(out[r], v) : out[r] + v;
        }
    return DG_OK;
}

int dg_rhs_adjoint(dg_ctx *c, const void *U, const double *w, double *ubar) {
    if (!c || !U || !w || !ubar || (const void *)ubar == U || ubar == w) return DG_EINVAL;
    if (c->fp32 || !c->LA || c->diff || c->sponge) return DG_ENOTIMPL;
    if (!c->base_set) return DG_ESTATE;
    DeviceGuard dg(c->device);
    int st = ensure_adjoint(c);
    if (st != DG_OK) return st;
    return rhs_adjoint_into(c, U, w, ubar, 0.0, 0.0, 1.0);
}

int dg_adjoint_step(dg_ctx *c, double dt, const void *U_n, const double *lam_np1, double *lam_n) {
    if (!c || !U_n || !lam_np1 || !lam_n || !std::isfinite(dt)) return DG_EINVAL;
    if ((const void *)lam_n == U_n || lam_n == lam_np1) return DG_EINVAL;
    if (c->fp32 || !c->LA || c->diff || c->sponge) return DG_ENOTIMPL;
    if (!c->base_set) return DG_ESTATE;
    DeviceGuard dg(c->device);
    int st = ensure_adjoint(c);
    if (st != DG_OK) return st;
    c->derived_valid = false;
    // forward stages of SSPRK(4,3) from U^n (Shu-Osher form):
    //   U1 = U^n + dt/2 R(U^n); U2 = U1 + dt/2 R(U1); U3 = 2/3 U^n + 1/3 U2 + dt/6 R(U2)
    void *X1 = c->adjX[0], *X2 = c->adjX[1], *X3 = c->adjX[2];
    st = prepare(c, U_n, 0);
    if (st == DG_OK) st = stage(c, MODE_STAGE, U_n, U_n, X1, 0, 0.0, 1.0, 0.5 * dt);
    if (st == DG_OK) st = stage(c, MODE_STAGE, X1, X1, X2, 1, 0.0, 1.0, 0.5 * dt);
    if (st == DG_OK) st = stage(c, MODE_STAGE, X2, U_n, X3, 0, 2.0 / 3.0, 1.0 / 3.0, dt / 6.0);
    if (st != DG_OK) return st;
    // reverse: U^{n+1} = U3 + dt/2 R(U3)
    double *l3 = c->adjL[0], *l2 = c->adjL[1], *l1 = c->adjL[2];
    st = rhs_adjoint_into(c, X3, lam_np1, l3, 0.0, 1.0, 0.5 * dt);            // l3 = l + dt/2 J3^T l
    if (st == DG_OK) st = rhs_adjoint_into(c, X2, l3, l2, 0.0, 1.0 / 3.0, dt / 6.0);  // l2
    if (st == DG_OK) st = rhs_adjoint_into(c, X1, l2, l1, 0.0, 1.0, 0.5 * dt);        // l1
    if (st != DG_OK) return st;
    // lam_n = 2/3 l3 + l1 + dt/2 J(U^n)^T l1
    const size_t bytes = (size_t)c->nodes * c->nf * sizeof(double);
    if (cudaMemcpyAsync(lam_n, l3, bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        return DG_ECUDA;
    return rhs_adjoint_into(c, U_n, l1, lam_n, 2.0 / 3.0, 1.0, 0.5 * dt);
}

int dg_cloud_functional(dg_ctx *c, const void *U, double *J, double *dJdU) {
    if (!c || !U || !J || !dJdU || (const void *)dJdU == U) return DG_EINVAL;
    if (c->fp32 || !c->LA) return DG_ENOTIMPL;
    if (!c->base_set) return DG_ESTATE;
    DeviceGuard dg(c->device);
    c->derived_valid = false;
    int st = prepare(c, U, 0);
    if (st != DG_OK) return st;
    AdjArgs A = adj_args(c, U, nullptr, dJdU, 0.0, 0.0, 1.0);
    if (c->LA->cloud(A, c->partials, c->nred, c->stream) != cudaSuccess) return DG_ECUDA;
    std::vector<double> h(c->nred);
    if (cudaMemcpyAsync(h.data(), c->partials, sizeof(double) * c->nred, cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess)
        return DG_ECUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return DG_ECUDA;
    double sum = 0.0;
    for (int b = 0; b < c->nred; ++b) sum += h[b];
    *J = sum;
    return DG_OK;
}

int dg_set_stabilisation(dg_ctx *c, const dg_stabilisation *sp) {
    if (!c || !sp) return DG_EINVAL;
    const dg_stabilisation p = *sp;
    const dg_config &g = c->cfg;
    if (!std::isfinite(p.gamma) || p.gamma < 0.0) return DG_EINVAL;
    if (p.gamma > 0.0 && !(std::isfinite(p.sigma) && p.sigma > 0.0)) return DG_EINVAL;
    if (!(p.sponge_alpha >= 0.0 && p.sponge_alpha <= 1.0)) return DG_EINVAL;
    const double top = g.L[g.dim - 1];
    if (p.sponge_alpha > 0.0 && !(p.sponge_zd >= 0.0 && p.sponge_zd < top)) return DG_EINVAL;
    const bool diff = p.gamma > 0.0, sponge = p.sponge_alpha > 0.0;
    if (diff && !c->face_pass) return DG_ENOTIMPL;
    if (c->in_ensemble && (diff || sponge)) return DG_ENOTIMPL;
    DeviceGuard dg(c->device);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return DG_ECUDA;
    MeshData &M = c->M;
    int st = DG_OK;
    if (diff && !c->alphaK) {
        // buffers of the diffusion: alpha per element and vertex, derivative
        // traces, a face-pass buffer with the symmetry terms
        const long long nvt = (long long)M.nv[0] * M.nv[1] * (g.dim == 3 ? M.nv[2] : 1);
        const size_t dtr = (size_t)2 * g.dim * c->nf * c->ne * c->nfp1 * c->rsz;
        st = alloc(c, &c->alphaK, (size_t)2 * c->ne * c->rsz);
        if (st == DG_OK) st = alloc(c, &c->alphaV, (size_t)2 * nvt * c->rsz);
        if (st == DG_OK) st = alloc(c, &c->dtrace[0], dtr);
        if (st == DG_OK) st = alloc(c, &c->dtrace[1], dtr);
        if (st == DG_OK) {
            const long long len = set_face_layout(c, 2 * c->nf);
            void *nb = nullptr;
            st = alloc(c, &nb, (size_t)len * c->rsz);
            if (st == DG_OK) {
                cudaFree(c->fbuf);
                c->device_bytes -= (size_t)(len / 2) * c->rsz;
                c->fbuf = nb;
            } else {
                set_face_layout(c, c->nf);
            }
        }
        if (st != DG_OK) return st;
    }
    if (diff) {
        const double h = std::pow(M.h[0] * M.h[1] * (g.dim == 3 ? M.h[2] : 1.0), 1.0 / g.dim);
        M.alpha_pre = p.gamma * 0.5 * std::pow(h, 1.0 - 0.5 * g.dim);
        for (int j = 0; j < 3; ++j)
            M.sigma_pen[j] = j < g.dim ? p.sigma * g.order * g.order / M.h[j] : 0.0;
        mesh_float_copies(M);
    }
    if (c->alphaK) set_face_layout(c, diff ? 2 * c->nf : c->nf);
    // sponge profile delta_R at the node levels (Section 3.6)
    if (sponge) {
        if (!c->sponge) st = alloc(c, &c->sponge, (size_t)M.nzlev_node * c->rsz);
        if (st != DG_OK) return st;
        std::vector<double> d(M.nzlev_node);
        for (int l = 0; l < M.nzlev_node; ++l) {
            const double z = c->z_node[l];
            d[l] = z >= p.sponge_zd
                       ? 0.5 * p.sponge_alpha * (1.0 - std::cos(M_PI * (z - p.sponge_zd) / (top - p.sponge_zd)))
                       : 0.0;
        }
        cudaError_t e;
        if (c->fp32) {
            std::vector<float> f(d.begin(), d.end());
            e = cudaMemcpy(c->sponge, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice);
        } else {
            e = cudaMemcpy(c->sponge, d.data(), sizeof(double) * d.size(), cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) return DG_ECUDA;
    } else if (c->sponge) {
        cudaFree(c->sponge);
        c->device_bytes -= (size_t)M.nzlev_node * c->rsz;
        c->sponge = nullptr;
    }
    c->stab = p;
    c->diff = diff;
    // alpha_K and the derivative traces come with the next split
    c->derived_valid = false;
    return DG_OK;
}

}  // extern "C"
