/*
 * dgmoist.h -- C interface of the GB300 library for the moist compressible
 * Euler discontinuous Galerkin method with implicit condensation
 * (Hittmeir, Lederer, Schoeberl, von Wahl, arXiv 2305.13847).
 *
 * What the library computes (the hot path of the method):
 *   - the pointwise implicit-condensation split, Eq. (2.8) solved by Newton's
 *     method at every node (Section 3.4);
 *   - the explicit DG right-hand side of Eq. (3.2)/(3.3): volume integrals of
 *     the flux of Eq. (2.11), Lax-Friedrichs face fluxes with the wave-speed
 *     bound Eq. (3.4) and slip-wall / periodic boundaries (Section 3.2), the
 *     warm-rain sources Eq. (2.4) and gravity, times the diagonal inverse mass
 *     matrix (Section 3.3);
 *   - the four-stage third-order SSP Runge-Kutta update (Remark 3.1).
 *
 * Discretisation conventions (fixed by this interface):
 *   - Structured Cartesian mesh of n[0] x n[1] (x n[2]) quadrilaterals /
 *     hexahedra on [0,L0] x [0,L1] (x [0,L2]).  The vertical direction is the
 *     last one (y in 2-D, z in 3-D); it always has slip walls at the bottom
 *     and top, the other directions are periodic or walls by periodic_mask.
 *   - Q^k space, k = order in 1..5, nodal basis at the (k+1) Gauss-Legendre
 *     points per direction; integrals by the same Gauss rule (collocation),
 *     so the mass matrix is exactly diagonal.
 *   - Unknowns U = (rho_d', rho_m', [rho_r'], m_0..m_{d-1}, E'), n_f = 3+d
 *     fields without rain and 4+d with rain: perturbations of the dry and
 *     moist (vapour + cloud) densities, rain density, momentum, perturbation
 *     of the total energy (Section 2.3, Eq. (2.11)).
 *   - "ABI layout" of a state: U[f][e][a], f the field, e = i0 + n0 (i1 + n1 i2)
 *     the element, a = a0 + (k+1)(a1 + (k+1) a2) the node (first index
 *     fastest).  Element storage type: double for DG_FP64 and DG_FP64_FFC,
 *     float for DG_FP32_BULK and DG_FP32_PERT.
 *   - Base (hydrostatic) state tables, Section 2.3: rho_d, rho_m, E, p at the
 *     node z-levels (index i_vert (k+1) + a_vert, n_vert (k+1) levels) and at
 *     the face z-levels (index i_vert, n_vert + 1 levels), as float64.
 *
 * Memory and ownership:
 *   - A context owns its device state, scratch buffers and stream binding.
 *     Pointers passed in are never freed or kept after the call returns.
 *   - "Device" pointers must point to memory on the context's current CUDA
 *     device; "host" pointers are ordinary host memory (pinned or pageable).
 *   - Work is enqueued on the CUDA stream given to dg_init_mesh (NULL = the
 *     legacy default stream).  Calls documented as synchronising wait for that
 *     stream before returning.
 *
 * Errors: every int-returning call returns DG_OK (0) or a negative code;
 * dg_strerror() describes it.  No call aborts or traps the device: the
 * kernels count Newton failures and non-physical states in device counters
 * that the synchronising calls turn into DG_ENOCONV / DG_ENONPHYS.
 */
#ifndef DGMOIST_H
#define DGMOIST_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DG_OK 0
#define DG_EINVAL (-1)   /* bad argument or size */
#define DG_ENOMEM (-2)   /* device allocation failed */
#define DG_ECUDA (-3)    /* a CUDA call failed */
#define DG_ENOCONV (-4)  /* Newton split hit its iteration cap somewhere */
#define DG_ENONPHYS (-5) /* non-physical or non-finite state (T, rho <= 0, NaN) */
#define DG_ESTATE (-6)   /* call order: base state or state not set yet */
#define DG_ENOTIMPL (-7) /* not implemented for this configuration */

#define DG_FP64 0
#define DG_FP32_BULK 1
#define DG_FP32_PERT 2
#define DG_FP64_FFC 3

#define DG_HOST 0
#define DG_DEVICE 1

/* Number of values written by dg_reduce. */
#define DG_NREDUCE 9

typedef struct dg_ctx dg_ctx;

typedef struct dg_config {
    int dim;            /* 2 or 3 */
    int n[3];           /* elements per direction (n[2] unused for dim 2), each >= 1 */
    int order;          /* polynomial degree k, 1..5 */
    double L[3];        /* domain lengths in m (L[2] unused for dim 2) */
    int periodic_mask;  /* bit j set: direction j periodic; the vertical is always walls */
    int rain;           /* 0: no rain (3+d fields); 1: warm rain (4+d fields) */
    int precision;      /* DG_FP64; DG_FP32_BULK: float state and flux arithmetic,
                           float64 split / temperature recovery / reductions;
                           DG_FP32_PERT: float throughout, the split solved in
                           the perturbation variables T - T_bar, rho_v - rho_v_bar
                           against a float64 split of the base state (no
                           cancellation, so float32 suffices there);
                           DG_FP64_FFC: float64 state and arithmetic as
                           DG_FP64, except that the stage kernel's volume
                           term and lift (the sum-factorised contractions of
                           Eq. (3.2) and the facet term of Eq. (3.3)) are
                           compensated float32-pair sums (error-free
                           transformations, ~2^-48 relative to the sum of the
                           terms' magnitudes) on the float32 pipe, which runs
                           64x the float64 rate on GB300; not in the paper */
    double g;           /* gravity in m/s^2 (the paper does not print it; 9.81 usual) */
    double rho_w;       /* water density in the rain speed: <= 0 takes the paper's
                           rho_w = rho_v + rho_c + rho_r; > 0 a constant (kg/m^3) */
    int faces;          /* where the Lax-Friedrichs face fluxes of a stage are
                           evaluated: DG_FACES_AUTO (0) the library's choice (the
                           face pass); DG_FACES_INLINE in the stage kernel, by both
                           elements of a face; DG_FACES_PASS once per face point in a
                           separate face kernel (an extra flux buffer of
                           n_f (k+1)^(d-1) values per face); DG_FACES_COLUMN (float32
                           forms only) in one kernel that marches each brick of
                           element columns upward and keeps the faces between
                           its elements on chip, only the brick sides' traces
                           passing through device memory.  The results agree to
                           rounding (float32 forms: bitwise); in every schedule
                           the two sides of a face get exactly opposite fluxes. */
} dg_config;

#define DG_FACES_AUTO 0
#define DG_FACES_INLINE 1
#define DG_FACES_PASS 2
#define DG_FACES_COLUMN 3

typedef struct dg_info {
    int n_fields;               /* n_f */
    int nodes_per_elem;         /* (k+1)^d */
    int face_points_per_face;   /* (k+1)^(d-1) */
    int n_zlev_node;            /* n_vert (k+1) */
    int n_zlev_face;            /* n_vert + 1 */
    int elems_per_block;        /* elements handled by one CTA of the stage kernel */
    long long n_elem;
    long long n_nodes;          /* n_elem * nodes_per_elem */
    long long n_dofs;           /* n_nodes * n_fields (the paper's DOF count) */
    size_t state_bytes;         /* bytes of one state in ABI layout */
    size_t device_bytes;        /* device memory held by the context */
    int launches_per_stage;     /* kernels per SSPRK stage: 1 (faces in the stage
                                   kernel) or 2 (face pass + stage kernel) */
} dg_info;

/* Warm-bubble workload: hydrostatic column of constant dry potential
 * temperature theta, surface pressure p_s, total-water mixing ratio
 * qt0 (1 - z/H), and a cos^2 potential-temperature bubble of the given
 * amplitude, centre and radii applied at fixed pressure and mixing ratio. */
typedef struct dg_bubble {
    double theta, p_s, qt0, H;
    double amplitude;
    double centre[3];
    double radius[3];
} dg_bubble;

/* Create a context for the mesh of cfg on the current CUDA device; work goes
 * to cuda_stream (a cudaStream_t, NULL for the default stream).  Allocates the
 * device state (two copies), derived fields and face-trace buffers.
 * Errors: DG_EINVAL for out-of-range fields or a mesh whose
 * n_nodes * n_fields exceeds 2^31 - 1; DG_ENOTIMPL for DG_FACES_COLUMN with
 * DG_FP64 or DG_FP64_FFC; DG_ENOMEM; DG_ECUDA. */
int dg_init_mesh(dg_ctx **out, const dg_config *cfg, void *cuda_stream);

/* Release everything owned by ctx (NULL is ignored). */
void dg_free(dg_ctx *ctx);

/* Sizes of the context's mesh and buffers. */
int dg_get_info(const dg_ctx *ctx, dg_info *info);

/* The library's Gauss-Legendre rule: n points in (-1, 1), ascending, and
 * weights, written to host arrays x[n], w[n]; n in 1..6.  Host only. */
int dg_gauss_legendre(int n, double *x, double *w);

/* Node and face z-levels of ctx's mesh in m, host arrays of
 * n_zlev_node and n_zlev_face entries. */
int dg_zlevels(const dg_ctx *ctx, double *z_node, double *z_face);

/* Set the hydrostatic base state (Section 2.3, Eq. (2.9)-(2.10)) from host
 * tables node_tab[4][n_zlev_node] and face_tab[4][n_zlev_face], rows
 * rho_d, rho_m, E, p (float64).  Copied; marks the derived fields stale. */
int dg_set_base_state(dg_ctx *ctx, const double *node_tab, const double *face_tab);

/* Build the warm-bubble workload in the context: base state tables
 * (hydrostatic column integrated with classical RK4, steps <= 1 m, on the
 * host) and the initial unknowns on the device (u = 0, rho_r' = 0).
 * noise: optional per-node temperature change in K, ABI node order
 * [e][a], float64, on host (where = DG_HOST) or device (DG_DEVICE); NULL for
 * none.  Errors: DG_EINVAL. */
int dg_init_bubble(dg_ctx *ctx, const dg_bubble *spec, const double *noise, int where);

/* Copy a state (ABI layout, the context's storage type) into / out of the
 * context.  where = DG_HOST or DG_DEVICE.  dg_set_state from DG_HOST with
 * the base state already set uploads in 8 chunks of whole element tiles on
 * a second stream of the context and splits each chunk (Eq. (2.8), the
 * derived fields and face traces the next step starts from) while the next
 * one uploads; otherwise it copies on the context's stream and the next
 * dg_step splits the state first.  Either way the results of later calls
 * are the same.  Both are asynchronous except dg_get_state with DG_HOST,
 * which synchronises; the host buffer of a DG_HOST upload must stay
 * unchanged until the stream has passed the call (pinned memory for an
 * asynchronous copy).  The split's Newton and non-physical counters
 * accumulate into dg_check_status as in dg_step.  Errors: DG_EINVAL,
 * DG_ESTATE (get before any set), DG_ECUDA. */
int dg_set_state(dg_ctx *ctx, const void *U, int where);
int dg_get_state(dg_ctx *ctx, void *U, int where);

/* Implicit-condensation split, Eq. (2.8), at every node of the state U
 * (device, ABI layout, storage type): writes float64 device arrays of
 * n_nodes values in [e][a] order -- T (K), rho_v, rho_c (kg/m^3) and
 * p_prime = (rho_d R_d + rho_v R_v) T - p_bar (Pa); any output may be NULL.
 * If n_unconverged is not NULL the call synchronises and stores the number
 * of nodes whose Newton iteration hit its cap.  Errors: DG_ESTATE without a
 * base state; DG_ENONPHYS if a non-physical node was found (synchronising
 * form only). */
int dg_saturation_split(dg_ctx *ctx, const void *U, double *T, double *rho_v,
                        double *rho_c, double *p_prime, long long *n_unconverged);

/* Semi-discrete right-hand side dU/dt = M^{-1}(-F(U) + G(U)), Eq. (3.5)-(3.6),
 * of the state U (device, ABI layout) into dUdt (device, ABI layout, the
 * storage type).  U and dUdt must not overlap.  Asynchronous. */
int dg_rhs(dg_ctx *ctx, const void *U, void *dUdt);

/* Advance the context's state by nsteps SSPRK(4,3) steps of size dt (s).
 * Synchronises at the end and returns DG_ENOCONV / DG_ENONPHYS if any node
 * failed during the call (the state is still advanced). */
int dg_step(dg_ctx *ctx, double dt, int nsteps);

/* dg_step followed by dg_get_state(ctx, U, DG_HOST), with the download
 * overlapping the last stage: the stage kernel of the final stage runs in
 * 8 chunks of whole element tiles, and each chunk's values are copied to
 * U (host, ABI layout, the storage type; pinned memory for a copy that
 * overlaps) on the context's second stream as soon as the chunk is done.
 * The state and U equal those of dg_step + dg_get_state bitwise.
 * nsteps >= 1.  Synchronises; returns dg_step's status.  Errors:
 * DG_EINVAL, DG_ESTATE, DG_ECUDA, DG_ENOCONV, DG_ENONPHYS. */
int dg_step_to_host(dg_ctx *ctx, double dt, int nsteps, void *U);

/* Same as dg_step but enqueues only: no synchronisation and no status
 * check (read it later with dg_check_status). */
int dg_step_async(dg_ctx *ctx, double dt, int nsteps);

/* Iteration cap of the Newton loops of the split Eq. (2.8) (Section 3.4) in
 * the following calls on ctx: max_iterations in 1..1000, default 50.  A node
 * whose iteration reaches the cap keeps its last iterate and is counted as
 * not converged (DG_ENOCONV from the synchronising calls).  Host setting, no
 * device work; an ensemble member takes it at the next dg_ensemble_configure.
 * Errors: DG_EINVAL. */
int dg_set_newton_limit(dg_ctx *ctx, int max_iterations);

/* Synchronise the stream and report (and clear) the failure counters
 * accumulated since the last check: DG_OK, DG_ENOCONV or DG_ENONPHYS.
 * counts (may be NULL) receives {n_unconverged, n_nonphysical}. */
int dg_check_status(dg_ctx *ctx, long long counts[2]);

/* Diagnostics of the context's state (synchronising), float64:
 *   out[0] integral of rho_d'            (dry-air mass perturbation)
 *   out[1] integral of rho_m' + rho_r'   (water mass perturbation)
 *   out[2] integral of m_0               (x-momentum)
 *   out[3] integral of rho_c             (cloud water)
 *   out[4] integral of rho_r'            (rain water; 0 without rain)
 *   out[5] max over nodes of |u| + v_r + c_m (for a CFL time step)
 *   out[6] max over nodes of (rho_v - rho_vs(T)) / rho_vs(T) (supersaturation)
 *   out[7] integral of E'
 *   out[8] rain fall-out: the water (rho_m + rho_r) that has left through
 *          the bottom and top walls since the state was last set
 *          (dg_set_state, dg_init_bubble), i.e. the time integral of the
 *          outward Lax-Friedrichs water flux over the wall faces, each
 *          stage weighted by its share of the step (dt/6, dt/6, dt/6, dt/2).
 *          The microphysics only moves water between rho_m and rho_r and
 *          interior faces cancel, so out[1] + out[8] is constant over
 *          dg_step calls up to rounding (Section 3.6's mass conservation,
 *          the rain examples of Section 4); the sponge layer, which turns
 *          moisture into dry air, breaks that balance.  0 without rain.
 * Integrals use the Gauss rule of the DG space (the diagonal mass matrix). */
int dg_reduce(dg_ctx *ctx, double out[DG_NREDUCE]);

/* Size of the fixed device scratch array used by dg_rhs_noalloc (32 MiB). */
#define DG_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* dg_rhs without any device allocation.  No counterpart in the paper: the
 * arithmetic is that of dg_rhs's kernels with the face fluxes evaluated
 * inside the stage kernel (the DG_FACES_INLINE schedule), so the result
 * agrees with dg_rhs to rounding; only where its scratch lives differs.
 *
 * For callers that cannot call cudaMalloc -- a host program whose memory
 * pool owns all device memory (a stray allocation would fragment it or
 * escape its accounting), a latency-critical loop that cannot pay for the
 * device synchronisation an allocation may imply, a process with a
 * device-memory budget fixed at start-up.  No context is needed: cfg
 * describes the mesh (precision must be DG_FP64, faces DG_FACES_AUTO or
 * DG_FACES_INLINE), base_node[4][n_zlev_node] and base_face[4][n_zlev_face]
 * are the base-state tables (device, float64, rows rho_d, rho_m, E, p,
 * levels as in dg_zlevels), U the state and dUdt the output (device, ABI
 * layout, float64, not overlapping).  Work goes to cuda_stream (a
 * cudaStream_t, NULL = default stream); the call is asynchronous and
 * allocates nothing: its scratch (saturation-density table, failure
 * counters, derived fields, face traces) is one file-scope device array of
 * DG_STATIC_SCRATCH_BYTES that each GPU loading the library holds until the
 * process exits.  The first call on a device (this one or
 * dg_rhs_noalloc_status) sets the array up with that device current -- looks
 * up its address, fills the table, zeroes the counters, and waits for that
 * work on the legacy default stream -- so make that first call before any
 * stream capture.  cudaDeviceReset invalidates the set-up: do not use these
 * entry points on a device after resetting it.  Every call shares the one
 * array, so calls whose work overlaps on the GPU (different streams,
 * different host threads) race; serialise them.  Newton iterations that hit
 * their cap and non-physical nodes are counted in the array across calls;
 * read them with dg_rhs_noalloc_status.
 * Errors: DG_EINVAL for a bad argument, a non-float64 precision, the face
 * pass, or a mesh whose scratch (derived fields + face traces) exceeds
 * DG_STATIC_SCRATCH_BYTES (e.g. about 1,800 elements of 3-D Q4 with rain);
 * DG_ECUDA. */
int dg_rhs_noalloc(const dg_config *cfg, const double *base_node, const double *base_face,
                   const void *U, void *dUdt, void *cuda_stream);

/* Failure counters of the dg_rhs_noalloc calls on the current device since
 * the last read: copies {n_unconverged, n_nonphysical} into counts (may be
 * NULL) and clears them, in order on cuda_stream, then synchronises that
 * stream.  Returns DG_ENONPHYS if any node was non-physical, else
 * DG_ENOCONV if a Newton iteration hit its cap, else DG_OK; DG_ECUDA.
 * Allocates nothing. */
int dg_rhs_noalloc_status(long long counts[2], void *cuda_stream);

/* Adjoint of the right-hand side: ubar = (dR/dU)^T w for R = dg_rhs at the
 * state U (device, ABI layout, float64), w and ubar device float64 arrays in
 * the ABI layout (ubar must not overlap U or w).  This is the linearisation
 * of the computed operator of Eq. (3.2)/(3.3): transposed volume
 * contraction and lift, Lax-Friedrichs flux with the active side of the max
 * in Eq. (3.4), and the split Eq. (2.8) differentiated by the implicit
 * function theorem on its active branch (saturated or not).  The fractional
 * powers of rain in v_r and in the warm-rain sources (Eq. (2.4)) have
 * unbounded derivatives as rho_r -> 0+; they are differentiated at
 * max(rho_r, 1e-12 kg/m^3), which keeps the linearisation of long runs
 * bounded and leaves it exact wherever rho_r >= 1e-12.  Uses the context's
 * derived-field and trace buffers (the next dg_step re-derives them).
 * DG_ENOTIMPL for float32 contexts (DG_FP32_BULK, DG_FP32_PERT);
 * asynchronous.  In a DG_FP64_FFC context the adjoint kernels are the
 * float64 ones. */
int dg_rhs_adjoint(dg_ctx *ctx, const void *U, const double *w, double *ubar);

/* Adjoint of one SSPRK(4,3) step of size dt from the state U_n (device,
 * ABI layout, float64): lam_n = (dU^{n+1}/dU^n)^T lam_np1.  The three
 * intermediate stage states are recomputed from U_n inside the call; the
 * stages are then reversed (Remark 3.1, Shu-Osher form) with dg_rhs_adjoint.
 * lam_np1, lam_n: device float64, ABI layout, distinct.  Allocates six
 * state-sized and one trace-sized scratch buffers in the context on first
 * use.  DG_ENOTIMPL for float32 contexts (DG_FP32_BULK, DG_FP32_PERT);
 * asynchronous.  A DG_FP64_FFC context recomputes the stage states with its
 * own stage kernel (float-float contractions). */
int dg_adjoint_step(dg_ctx *ctx, double dt, const void *U_n, const double *lam_np1,
                    double *lam_n);

/* Cloud-water functional J(U) = integral of rho_c = rho_m - rho_v over the
 * domain (Gauss rule of the DG space; rho_v from the split Eq. (2.8)) and
 * its gradient dJ/dU (device float64, ABI layout).  J is written to a host
 * double; the call synchronises.  DG_ENOTIMPL for float32 contexts
 * (DG_FP32_BULK, DG_FP32_PERT). */
int dg_cloud_functional(dg_ctx *ctx, const void *U, double *J, double *dJdU);

/* ---- Stabilisation: artificial diffusion and sponge layer ----------------
 *
 * Artificial diffusion (Section 3.5, Eq. (3.7)): every field of U gets the
 * symmetric interior-penalty form with a continuous coefficient alpha:
 * per element alpha_K = gamma 0.5 h^(1-d/2) ||w||_{0,K} (h = |K|^(1/d);
 * w = u, or u - v_r e_z for rho_r), projected to continuous Q1 by averaging
 * over the elements at each vertex; penalty sigma k^2 / h_j on interior
 * faces (walls carry no diffusive flux).  The coefficient follows the state
 * the right-hand side is evaluated on.  Needs the face pass (dg_config.faces
 * == DG_FACES_AUTO or DG_FACES_PASS).
 *
 * Sponge (Section 3.6, Eq. (3.8)), after every dg_step step:
 * rho_m', rho_r', m, E' <- (1 - delta) (.) and rho_d' += delta (rho_m' + rho_r')
 * at every node, delta = alpha/2 (1 - cos(pi (z - z_D)/(z_top - z_D))) above
 * z_D, 0 below. */
typedef struct dg_stabilisation {
    double gamma;         /* diffusion scale; 0 switches the diffusion off */
    double sigma;         /* interior-penalty parameter (> 0 when gamma > 0), e.g. 10 */
    double sponge_zd;     /* bottom of the sponge layer in m, 0 <= z_D < top */
    double sponge_alpha;  /* sponge strength in [0, 1]; 0 switches it off */
} dg_stabilisation;

/* Set (or clear, with zeros) the stabilisation of ctx for the following
 * dg_rhs / dg_step calls; allocates the diffusion buffers on first use.
 * Synchronises ctx's stream.  Errors: DG_EINVAL for out-of-range values;
 * DG_ENOTIMPL for diffusion without the face pass or for an ensemble member;
 * DG_ENOMEM; DG_ECUDA.  dg_rhs_adjoint and dg_adjoint_step return
 * DG_ENOTIMPL while either term is on. */
int dg_set_stabilisation(dg_ctx *ctx, const dg_stabilisation *s);

/* ---- Batched ensemble (not in the paper, which runs one case at a time) ----
 * Many independent 2-D meshes (any sizes, orders 1..5, rain on or off),
 * FP32-bulk, advanced together.  One step is captured in a CUDA graph and
 * replayed, in one of two schedules:
 *  - persistent (dg_ensemble_configure): each SSPRK(4,3) stage is one
 *    persistent launch whose CTAs take element tiles of any member from an
 *    atomic work counter and run the single-mesh stage code for that
 *    member's order, with the face fluxes evaluated in the tile;
 *  - branches (dg_ensemble_configure_branches): each member's step is
 *    dg_step's own launches (face pass, then stage, four times), and the
 *    members form parallel branches of the graph.
 * Results are bitwise those of dg_step on each member in both. */
typedef struct dg_ensemble dg_ensemble;

/* Create n members (cfgs[i].dim == 2, precision DG_FP32_BULK or DG_FP32_PERT) and build
 * each one's warm bubble (dg_init_bubble with bubbles[i], no noise).  Work
 * goes to cuda_stream, which must not be the legacy default stream (the
 * steps are captured in a graph); NULL creates a private stream.
 * Errors: DG_EINVAL, DG_ENOMEM, DG_ECUDA. */
int dg_ensemble_create(dg_ensemble **out, int n, const dg_config *cfgs, const dg_bubble *bubbles,
                       void *cuda_stream);

/* Member i's context (owned by the ensemble; use it for dg_get_state,
 * dg_reduce, ...; do not free it). */
int dg_ensemble_member(dg_ensemble *ens, int i, dg_ctx **ctx);

/* Total DOFs over all members. */
long long dg_ensemble_dofs(const dg_ensemble *ens);

/* Set the members' time steps dt[n] (s, host) and the launch shape:
 * blocks_per_sm persistent CTAs per SM (capped by occupancy), the order of
 * work items (0 member by member, 1 round-robin over members, 2 largest
 * members first), the register budget regs (0: 128 registers per thread,
 * two CTAs per SM; 1: 80 registers, three CTAs per SM) and tiles_per_item
 * (1..64) element tiles of one member per work item (a CTA takes that many
 * consecutive tiles at once: fewer queue operations and barriers per
 * element, coarser balance); re-derives each member's split and traces if
 * needed and re-captures the step graph.  Synchronises. */
int dg_ensemble_configure(dg_ensemble *ens, const double *dt, int blocks_per_sm, int item_order,
                          int regs, int tiles_per_item);

/* Set the members' time steps dt[n] (s, host) and capture the branch
 * schedule: members are dealt, largest first, to `lanes` (>= 1; capped at
 * n) parallel branches, each member to the branch with the fewest DOFs so
 * far; a branch steps its members one after another.  Every member must
 * use the face pass (created with DG_FACES_AUTO or DG_FACES_PASS), else
 * DG_EINVAL.  Re-derives each member's split and traces if needed.
 * Synchronises.  Errors: DG_EINVAL, DG_ECUDA. */
int dg_ensemble_configure_branches(dg_ensemble *ens, const double *dt, int lanes);

/* Persistent schedule: the grid size and the number of work items (element
 * tiles) of the captured step.  Branch schedule: the number of branches and
 * the number of members. */
int dg_ensemble_launch_shape(const dg_ensemble *ens, int *grid, int *n_items);

/* Replay the captured step nsteps times.  dg_ensemble_step synchronises and
 * returns the worst member status (DG_ENONPHYS before DG_ENOCONV);
 * dg_ensemble_step_async only enqueues.  DG_ESTATE before
 * dg_ensemble_configure or dg_ensemble_configure_branches. */
int dg_ensemble_step(dg_ensemble *ens, int nsteps);
int dg_ensemble_step_async(dg_ensemble *ens, int nsteps);

/* Free the ensemble and its members (NULL is ignored). */
void dg_ensemble_free(dg_ensemble *ens);

/* ---- Self-test of the library's float64 elementary functions -------------
 * Not part of the method (no counterpart in the paper): a verification aid.
 * The float64 kernels replace CUDA's conversions, divisions, square roots,
 * pow and exp/log on their hot paths by their own functions -- float32 <->
 * float64 conversions and compares on the bit pattern, Newton-Raphson
 * refinement of the hardware's approximate reciprocal and reciprocal square
 * root, one third-order step for r^(-1/16) and r^(-1/8) from a float32
 * estimate, a Taylor table for rho_vs(T) of Eq. (2.6).  dg_selftest_math
 * evaluates function fn of the library at the n float64 values x (device)
 * and writes, to out[4n] (device, float64):
 *   out[0 .. n)    the library's value,
 *   out[n .. 2n)   the value of the function it stands in for, computed by
 *                  CUDA: the hardware conversion (NARROW: float64 -> float32,
 *                  WIDEN: float32 -> float64 of the float32-rounded x), IEEE
 *                  division 1/x (RECIP), 1/sqrt(x) by IEEE sqrt and division
 *                  (RSQRT), IEEE sqrt (SQRT), pow(x, -1/16) (INV_ROOT16),
 *                  pow(x, -1/8) (INV_ROOT8), the closed form
 *                  e_s(T) / (R_v T) with exp and log (RHO_VS; RHO_VS_F32 takes
 *                  the float32-rounded temperature, the overload the float32
 *                  pre-solve uses; RHO_VS_BULK, at the float32-rounded
 *                  temperature too, is the value-only evaluation of the
 *                  FP32-bulk split, its curvature terms in float32), or for
 *                  COMPARE the bits of the plain
 *                  float64 compares x > 0, x > 1.5, x < 1.5, |x| <= 1.5,
 *                  isfinite(x), max(|x|, 1.5) against those of the library's
 *                  bit-pattern compares;
 *                  FF_SPLIT writes hi + lo of the float32 pair of
 *                  DG_FP64_FFC (in float64) and, beside it, x itself;
 *   out[2n .. 4n)  for FF_SPLIT the pair's hi and CUDA's float32 rounding
 *                  of x; for RHO_VS / RHO_VS_F32 / RHO_VS_BULK the derivative
 *                  d rho_vs / dT, the library's (RHO_VS_BULK: the float32
 *                  derivative that split forms) and the closed form's; 0
 *                  otherwise.
 * Uses ctx's rho_vs table and stream; synchronises.  Errors: DG_EINVAL
 * (bad fn or n, or a device other than ctx's current); DG_ECUDA. */
#define DG_MATH_NARROW 0
#define DG_MATH_WIDEN 1
#define DG_MATH_RECIP 2
#define DG_MATH_RSQRT 3
#define DG_MATH_SQRT 4
#define DG_MATH_INV_ROOT16 5
#define DG_MATH_INV_ROOT8 6
#define DG_MATH_RHO_VS 7
#define DG_MATH_RHO_VS_F32 8
#define DG_MATH_COMPARE 9
#define DG_MATH_RHO_VS_BULK 10
#define DG_MATH_FF_SPLIT 11
int dg_selftest_math(dg_ctx *ctx, int fn, const double *x, double *out, long long n);

/* Float64 FMA throughput probe (a measurement aid, not part of the method):
 * enqueues on cuda_stream one kernel of `blocks` CTAs x 256 threads, each
 * thread running 8 independent chains of `iters` dependent fmas, and writes
 * each thread's result to out[blocks * 256] (device, float64).  *flops (host,
 * may be NULL) receives the kernel's float64 operation count, 2 per fma, so
 * that the caller's timing of the launch gives the FP64 rate.  Asynchronous.
 * Errors: DG_EINVAL, DG_ECUDA. */
int dg_fp64_fma_probe(double *out, int blocks, long long iters, void *cuda_stream, double *flops);

/* Text for a status code. */
const char *dg_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* DGMOIST_H */
