/*
 * liblbm: GB300 (sm_103a) library for the per-time-step lattice update of the
 * thermal multiphase lattice Boltzmann method of Kupershtokh, Medvedev and
 * Gribanov, "Thermal lattice Boltzmann method for multiphase flows"
 * (arXiv:1705.10045).
 *
 * One time step (lbm_step) does, for every node of a D2Q9 or D3Q19 lattice:
 *   1. moments rho = sum N_k, rho u = sum c_k N_k (Eq. (hydro)), E = sum g_k,
 *      T = E/(rho c_v) (Sec. 4);
 *   2. van der Waals pressure p = kappa p~(rho, T), pseudopotential
 *      U = p - rho theta, Phi = sqrt(-U) (Sec. 3, Eq. (force));
 *   3. the mixed interparticle force of Sec. 3 (mixing parameter A, stencil
 *      weights G_k, alpha) plus gravity, du = F dt/rho, u* = u + du/2
 *      (Eq. (edm), Eq. (ustar));
 *   4. the finite-difference energy change dE = -p div(u*) + div(lambda grad T)
 *      (Sec. 4, Sec. 6.2);
 *   5. BGK collision + EDM source for N (Eq. (lbe), Eq. (edm)) and, for the
 *      energy populations g (Eq. (gk)), BGK + g dE/E + the energy pseudoforce
 *      g^eq(E, u+du) - g^eq(E, u) (Sec. 4);
 *   6. streaming to x + c_k, periodic, or halfway bounce-back at walls
 *      (per axis; each wall adiabatic or held at a fixed temperature through
 *      the conduction term).  The paper's runs are periodic; a wall is the
 *      halfway bounce-back of both population sets, and the stencils read
 *      the mirror node beyond it (Phi and rho as they are, the velocity
 *      component normal to the wall negated, T mirrored or reflected about
 *      the wall temperature).
 *
 * Lattice units: h = dt = 1, theta = 1/3.  Velocity ordering: k = 0 rest,
 * then nearest neighbours, then next-nearest, each direction followed by its
 * opposite (D2Q9: +x -x +y -y (+x+y) (-x-y) (+x-y) (-x+y); D3Q19: +x -x +y -y
 * +z -z, then the face diagonals (+x+y)(-x-y)(+x-y)(-x+y)(+x+z)(-x-z)(+x-z)
 * (-x+z)(+y+z)(-y-z)(+y-z)(-y+z)).
 *
 * Field layout for every array crossing this interface: structure of arrays,
 * x fastest: a scalar field is nx*ny*nz doubles indexed (z*ny + y)*nx + x
 * (nz = 1 for D2Q9); a vector field is d such planes (x component first).
 *
 * Errors: every call returns LBM_OK (0) or a negative LBM_ERR_* code and
 * leaves a message for lbm_last_error() (thread-local).  Device-side
 * problems (U >= 0 clamped, non-finite or non-positive density or energy)
 * are counted on the device and reported as LBM_ERR_NONPHYSICAL by the
 * next synchronising call (lbm_moments, lbm_diagnostics, lbm_sync,
 * lbm_get_state).  Calls on one handle are not thread-safe.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_ERR_INVALID_ARG (-1)
#define LBM_ERR_UNSTABLE_PARAMS (-2)
#define LBM_ERR_OOM (-3)
/* A CUDA call failed; the state of the steps since the last synchronising
 * call is then not valid. */
#define LBM_ERR_CUDA (-4)
#define LBM_ERR_NONPHYSICAL (-5)
/* A wait inside the fused step gave up: the warps of a CTA hand planes over
 * through shared-memory barriers whose waits are bounded to about half a
 * second, after which the CTA finishes without waiting and counts the
 * timeout.  Every synchronising call reports it until lbm_init or
 * lbm_set_state gives the handle a new state.  lbm_test_drop_handoff makes
 * such a wait run out on purpose (tests only). */
#define LBM_ERR_TIMEOUT (-6)

#define LBM_D2Q9 9
#define LBM_D3Q19 19

/* storage (and arithmetic) of the population sets */
#define LBM_STORE_FP64 0 /* FP64 storage, FP64 arithmetic */
#define LBM_STORE_FP32 1 /* FP32 storage, FP32 arithmetic */
#define LBM_STORE_FP16 2 /* FP16 storage of N_k - w_k rho_ref and g_k - w_k E_ref, FP32 arithmetic */

/* how a time step is launched: one fused kernel that marches CTA tiles along
 * the last lattice axis, or three kernels (moments/Phi, force, collide+stream)
 * with the fields in device memory; both compute the same step */
#define LBM_STEP_FUSED 0
#define LBM_STEP_THREE_LAUNCH 1

/* where a caller buffer lives */
#define LBM_MEM_HOST 0
#define LBM_MEM_DEVICE 1

typedef struct lbm_handle lbm_handle;

/* Parameters of one simulation domain.  Citations give the passage that
 * defines each quantity. */
typedef struct lbm_params {
    int lattice;          /* LBM_D2Q9 or LBM_D3Q19 (Sec. 2) */
    int nx, ny, nz;       /* lattice size; nz must be 1 for D2Q9 */
    double kappa;         /* lattice pressure scale: p = kappa p~(rho, T), reduced vdW
                             p~ = 8 rho T/(3 - rho) - 3 rho^2 (Sec. 3) */
    double A;             /* force mixing parameter (Sec. 3; -0.152 for vdW) */
    int barotropic;       /* nonzero: the EOS uses T0 instead of T (Sec. 4) */
    double T0;
    double tau;           /* relaxation time of N (Sec. 2), > 1/2 */
    double tau_E;         /* relaxation time of g (Eq. (gk)), > 1/2 */
    double c_v;           /* specific heat, E = rho c_v T (Sec. 4), > 0 */
    int chi_mode;         /* 0: constant conductivity lambda; 1: lambda = rho c_v chi (Sec. 4) */
    double lambda, chi;
    double gravity[3];    /* body force per unit mass, added to F (Sec. 2: F is the total force) */
    int wall;             /* last axis (y for D2Q9, z for D3Q19): 0 periodic, 1 bounce-back
                             walls beyond both ends */
    int T_fixed_lo, T_fixed_hi; /* per wall of the last axis: 0 adiabatic, 1 held at T_lo / T_hi */
    double T_lo, T_hi;
    int wall_x;           /* x axis: 0 periodic, 1 bounce-back walls beyond both ends */
    int wall_y;           /* y axis of D3Q19 (must be 0 for D2Q9, whose y is the last axis) */
    int T_fixed_x[2], T_fixed_y[2]; /* per wall (low, high end): 0 adiabatic, 1 held at T_x[i] / T_y[i] */
    double T_x[2], T_y[2];
    int pressure_work;    /* include -p div(u*) in dE (Sec. 4) */
    int conduction;       /* include div(lambda grad T) in dE (Sec. 4) */
    int pseudoforce;      /* include the energy pseudoforce (Sec. 4) */
    double latent;        /* rho_liq Q of Sec. 5, energy per volume in the units of
                             E = rho c_v T; 0 (default) switches the latent heat off.
                             When nonzero, dE gains -latent rho div(u*)/(rho_l - rho_v)
                             at nodes with rho_v(T) < rho < rho_l(T), the Maxwell
                             densities interpolated linearly in T on the grid
                             T = 0.5 + j/1024 (j = 0..512; T < 0.5 takes the first
                             point, T >= 1 has no transition layer) */
    int storage;          /* LBM_STORE_* */
    double rho_ref, E_ref;/* shifts of the FP16 storage (ignored otherwise) */
    int step_kernel;      /* LBM_STEP_FUSED (default) or LBM_STEP_THREE_LAUNCH */
    void* stream;         /* cudaStream_t the library enqueues on (NULL: default stream) */
    int device;           /* CUDA device ordinal */
} lbm_params;

/* Maxwell coexistence densities of the reduced vdW fluid at 0 < T < 1
 * (Sec. 3): equal pressure and chemical potential of the two phases.  Host
 * computation, no device needed.  Returns LBM_OK, or LBM_ERR_INVALID_ARG for
 * T outside (0, 1) or a null pointer. */
int lbm_coexistence(double T, double* rho_v, double* rho_l);

/* Fill *p with defaults: D2Q9 64x64x1, kappa 0.01, A -0.152, tau = tau_E = 1,
 * c_v 1.5, lambda 0.05, periodic, all physics switches on, FP32 storage,
 * rho_ref 1, E_ref 1.2, default stream, device 0. */
void lbm_default_params(lbm_params* p);

/* Validate *p, run the pre-flight checks (tau, tau_E > 1/2; c_v > 0;
 * kappa > 0; sizes >= 1 and nz == 1 for D2Q9; wall axis at least 2 nodes)
 * and allocate all device state on p->device.  The library owns that state
 * until lbm_destroy.  Errors: LBM_ERR_INVALID_ARG, LBM_ERR_OOM, LBM_ERR_CUDA. */
int lbm_create(const lbm_params* p, lbm_handle** out);

/* Set the populations to equilibrium: N = N^eq(rho, u), g = g^eq(rho eps, u)
 * (Eq. (feq)), where eps = c_v T is the specific internal energy and u is
 * taken as the lattice velocity of Eq. (hydro).  rho, eps: one plane each;
 * u: d planes.  mem says whether the three pointers are host or device
 * memory; the library copies them and does not keep them.  Rejects
 * rho <= 0, eps <= 0, non-finite values and U = p - rho theta >= 0
 * (LBM_ERR_NONPHYSICAL), and nodes breaking the stability criteria
 * (dp/drho)_T <= (h/dt)^2 + theta (Sec. 3) or chi dt/h^2 < 0.5/d (Sec. 6.1)
 * (LBM_ERR_UNSTABLE_PARAMS); the checks run on the device.  Host input goes
 * through a device staging buffer the handle keeps.  Resets the step
 * counter.  Synchronising. */
int lbm_init(lbm_handle* h, const double* rho, const double* u, const double* eps, int mem);

/* Enqueue n time steps on the handle's stream (asynchronous, n >= 0). */
int lbm_step(lbm_handle* h, int n);

/* Output fields of the current state: rho, the physical velocity u*
 * (Eq. (ustar), d planes), T = E/(rho c_v) and P = kappa p~(rho, T).  Any
 * pointer may be NULL.  mem: host or device.  Synchronising; returns a
 * latched device error if any. */
int lbm_moments(lbm_handle* h, double* rho, double* u, double* T, double* P, int mem);

/* FP32 twin of lbm_moments: the same fields, computed as lbm_moments does
 * and rounded to the nearest float (half the bytes to move).  Host output
 * is staged through the handle's second population buffer, which the next
 * step overwrites anyway.  Synchronising; errors as lbm_moments. */
int lbm_moments_f(lbm_handle* h, float* rho, float* u, float* T, float* P, int mem);

/* Global sums of the current state: each node's moments, formed in the
 * arithmetic type, summed in FP64 with Kahan compensation in a fixed order
 * (bitwise reproducible): out[0] mass, out[1..3] momentum
 * sum c_k N_k (x, y, z), out[4] internal energy, out[5] clamped nodes (U >= 0)
 * and out[6] non-finite or non-positive nodes since the last lbm_init,
 * out[7] steps taken since lbm_init.  Synchronising. */
int lbm_diagnostics(lbm_handle* h, double out[8]);

/* Size in bytes of the raw state for lbm_get_state / lbm_set_state: a
 * 16-byte header (magic "LBM1", lattice, storage, step count) followed by the
 * 2Q population planes N_0..N_{Q-1}, g_0..g_{Q-1} (each nx*ny*nz values, x
 * fastest) in the storage format.  On the device the library keeps the two
 * sets interleaved (for each k the node pairs (N_k, g_k)); lbm_get_state and
 * lbm_set_state convert, using the handle's idle population buffer. */
size_t lbm_state_bytes(const lbm_handle* h);

/* Copy the raw state out or in (checkpoint / resume; resuming is bitwise
 * identical to not stopping).  buf is host or device memory of
 * lbm_state_bytes bytes.  Synchronising. */
int lbm_get_state(lbm_handle* h, void* buf, int mem);
int lbm_set_state(lbm_handle* h, const void* buf, int mem);

/* Wait for the handle's stream; returns a latched device error if any. */
int lbm_sync(lbm_handle* h);

/* Number of kernel launches one lbm_step(1) enqueues. */
int lbm_launches_per_step(const lbm_handle* h);

/* Advance n >= 1 steps like lbm_step, with a CUDA event pair around every
 * launch on the handle's stream, and write the mean duration in ms of launch
 * j of a step to ms[j] for j < min(cap, launches).  Returns the number of
 * launches per step (> 0) or an LBM_ERR_* code.  Synchronising. */
int lbm_profile_step(lbm_handle* h, int n, double* ms, int cap);

/* Kernel name of launch j of a step ("" when out of range). */
const char* lbm_launch_name(const lbm_handle* h, int j);

/* Free all device state.  NULL is allowed. */
void lbm_destroy(lbm_handle* h);

/* ---------------------------------------------------------------------------
 * Batches: many independent domains (different sizes, same lattice and
 * storage) advanced together.  lbm_batch_step(n) is one persistent kernel
 * launch that covers every step of every domain through a table of
 * (domain, tile, chunk) work items: CTAs take (step, item) work in order from
 * a counter, and an item of step s of a domain starts once every item of that
 * domain has finished step s - 1 (per-domain completion counters in device
 * memory, waits bounded to about half a second, then LBM_ERR_TIMEOUT on that
 * domain).  The request (clearing the counters, the launch, the descriptor
 * bookkeeping) is captured in a CUDA graph and replayed.  Each domain keeps
 * its own state in its own device memory and has a step budget:
 * lbm_batch_step(n) advances every domain by min(n, its remaining budget)
 * steps, so jobs with different step counts share the launch.  Results are
 * bitwise identical to running each domain alone with lbm_step (the
 * per-node arithmetic is the same kernel code).  The paper has no
 * counterpart: this is the batched form of its per-step update for many
 * simulation jobs. */
typedef struct lbm_batch lbm_batch;

/* Device memory in bytes a domain with parameters *p needs (admission control),
 * counting the staging planes it keeps once fields have moved between it and
 * host memory (lbm_init or lbm_moments with host pointers). */
size_t lbm_domain_bytes(const lbm_params* p);

/* New empty batch for common->lattice and common->storage on common->device.
 * Work is enqueued on common->stream, or on a stream the batch creates when
 * it is NULL (graphs cannot be captured on the legacy default stream). */
int lbm_batch_create(const lbm_params* common, lbm_batch** out);

/* Create a domain with parameters *p (lattice and storage must match the
 * batch; stream and device are the batch's), initialise it from rho, u, eps
 * as lbm_init does, give it a budget of `steps` steps and return its slot id.
 * Errors as lbm_create and lbm_init (LBM_ERR_OOM when memory runs out). */
int lbm_batch_add(lbm_batch* b, const lbm_params* p, const double* rho, const double* u, const double* eps,
                  int mem, long long steps, int* id);

/* Destroy a domain and free its slot (synchronising). */
int lbm_batch_remove(lbm_batch* b, int id);

/* Enqueue n step launches; every domain takes min(n, budget) steps. */
int lbm_batch_step(lbm_batch* b, int n);

/* Steps a domain has taken since its initialisation and steps left in its budget. */
int lbm_batch_status(const lbm_batch* b, int id, long long* steps_done, long long* steps_left);

/* Set a domain's remaining budget. */
int lbm_batch_set_budget(lbm_batch* b, int id, long long steps);

/* The domain's handle, borrowed for lbm_moments, lbm_diagnostics,
 * lbm_get_state, lbm_sync (not lbm_destroy or lbm_step); NULL for a bad id. */
lbm_handle* lbm_batch_domain(lbm_batch* b, int id);

/* Number of domains in the batch. */
int lbm_batch_size(const lbm_batch* b);

/* CTA shapes the batch kernel can run with, their names, and selection. */
int lbm_batch_variants(const lbm_batch* b);
const char* lbm_batch_variant_name(const lbm_batch* b, int v);
int lbm_batch_set_variant(lbm_batch* b, int v);

/* Autotune: time `reps` launches of every CTA shape on the batch's current
 * domains (each launch writes a step into the spare buffers and leaves the
 * state and counters unchanged), keep the fastest, write its index to *best
 * and the mean ms per launch of shape v to ms[v] (ms may be NULL). */
int lbm_batch_tune(lbm_batch* b, int reps, int* best, double* ms);

/* Test hook, not for production runs: in the following lbm_batch_step
 * requests, work item `item` of the table (0-based) does not report the end
 * of its first step, so the next step's items of its domain wait until their
 * bounded wait runs out and that domain reports LBM_ERR_TIMEOUT (a separately
 * compiled instance of the batch kernel; the ordinary one has no trace of
 * it).  item < 0 switches it off.  Errors: LBM_ERR_INVALID_ARG for a null
 * batch. */
int lbm_batch_test_drop_item(lbm_batch* b, int item);

/* Wait for the batch's work; returns a latched device error of any domain. */
int lbm_batch_sync(lbm_batch* b);

/* Destroy every domain and the batch.  NULL is allowed. */
void lbm_batch_destroy(lbm_batch* b);

/* ---------------------------------------------------------------------------
 * Slabs: one domain cut along its last axis (y for D2Q9, z for D3Q19) into
 * `count` sub-domains that step independently and swap halo planes after
 * every step.  This is the decomposition a run over several GPUs needs (one
 * slab per GPU, the halo swap over the interconnect); within one process the
 * slabs live on one device and the swap is a device-to-device copy.  The
 * paper gives no parallel scheme; the halo depth follows from the reach of
 * one step along an axis: the collision of plane c reads the moments and the
 * velocity change du (Sec. 3, force with the stencil of Sec. 3, Eq. (edm))
 * of planes c-1..c+1, du reads Phi one plane further, and the finite
 * differences of Sec. 4 read planes c-1..c+1; so the collision of plane c
 * depends on planes c-2..c+2, and with LBM_SLAB_HALO = 2 halo planes beyond
 * each cut every plane a slab owns is collided exactly.  A slab collides its
 * owned planes only (lbm_set_step_planes); its edge planes push the
 * populations that cross a cut into its halo planes.  The swap after each
 * step does two things: (1) the crossing populations of each cut (the
 * directions whose velocity points across it, 5 for D3Q19 and 3 for D2Q9;
 * lbm_get_crossing / lbm_set_crossing) move from the pushing slab's halo
 * plane to the owning slab's edge plane; (2) each slab's halo planes are
 * overwritten with its neighbours' edge planes, complete after (1).  On one
 * GPU (lbm_slabs_*) these are two phases of device copies.  Between
 * processes they fit in one message per neighbour and direction: the
 * crossing populations and the two edge planes, where the receiver restores
 * its own crossing populations into the halo plane next to the cut (the
 * Python binding's SlabRank; with lbm_step_begin the planes next to the cuts
 * step first and the messages travel while the interior steps).
 * FP64 and FP32 slabs reproduce the undivided domain bit for bit; FP16 slabs
 * key their stochastic rounding by node index within the slab, so they agree
 * in distribution, not in bits. */
#define LBM_SLAB_HALO 2

typedef struct lbm_slab {
    int first;       /* first plane the slab owns, as an index of the whole domain's last axis */
    int own;         /* planes it owns: nm / count, plus one for the first nm % count slabs */
    int lo, hi;      /* halo planes below / above the owned ones: LBM_SLAB_HALO at a cut, 0 at a wall */
    int below, above;/* slab across the lower / upper cut (periodic domains wrap), -1 at a wall */
    lbm_params p;    /* the slab's own domain: last axis lo + own + hi planes; a fixed wall
                        temperature is kept only where the slab ends at the domain's wall */
} lbm_slab;

/* Host-only plan of slab i of `count` for the domain *p (no device needed).
 * Errors (LBM_ERR_INVALID_ARG): null pointers, unknown lattice, count < 1,
 * i outside [0, count), or slabs that would own fewer than LBM_SLAB_HALO
 * planes. */
int lbm_slab_plan(const lbm_params* p, int count, int i, lbm_slab* out);

typedef struct lbm_slabs lbm_slabs;

/* The domain *p as `count` slabs on p->device, all enqueued on p->stream
 * (count = 1 is the undivided domain).  The library owns the slab handles
 * and a field buffer of (d + 3) planes of doubles per node of the largest
 * slab.  Errors as lbm_slab_plan and lbm_create. */
int lbm_slabs_create(const lbm_params* p, int count, lbm_slabs** out);

/* Number of slabs (LBM_ERR_INVALID_ARG for NULL). */
int lbm_slabs_count(const lbm_slabs* s);

/* Handle of slab i (owned by the slabs object; NULL if out of range). */
lbm_handle* lbm_slabs_domain(lbm_slabs* s, int i);

/* As lbm_init for the whole domain's fields (same layout and checks); each
 * slab is initialised from its own and its halo planes.  Synchronising. */
int lbm_slabs_init(lbm_slabs* s, const double* rho, const double* u, const double* eps, int mem);

/* n steps: every slab steps once, then the two exchange rounds refresh every
 * halo, n times (asynchronous on p->stream). */
int lbm_slabs_step(lbm_slabs* s, int n);

/* As lbm_moments for the whole domain, assembled from the slabs' owned
 * planes.  Synchronising; LBM_ERR_NONPHYSICAL as lbm_moments. */
int lbm_slabs_moments(lbm_slabs* s, double* rho, double* u, double* T, double* P, int mem);

/* As lbm_diagnostics for the whole domain: the sums over each slab's owned
 * planes (FP64 with Kahan compensation per thread, across threads and across slabs
 * in slab order); out[5], out[6] add up the slabs' counters, halo planes
 * included; out[7] the steps since lbm_slabs_init.  Synchronising. */
int lbm_slabs_diagnostics(lbm_slabs* s, double out[8]);

/* Wait for every slab; returns a latched device error if any. */
int lbm_slabs_sync(lbm_slabs* s);

/* Free every slab handle and the field buffer.  NULL is allowed. */
void lbm_slabs_destroy(lbm_slabs* s);

/* Halo exchange between processes (one slab handle per process): bytes of one
 * plane of the last axis over all 2Q populations in the handle's storage
 * format. */
size_t lbm_plane_bytes(const lbm_handle* h);

/* Copy planes [first, first + count) of the current populations out of / into
 * buf in the device layout: Q rows (k = 0..Q-1) of count planes each, every
 * node a pair (N_k, g_k), storage format.  mem = LBM_MEM_DEVICE: one kernel on the handle's stream,
 * asynchronous (the caller orders its own use of buf on that stream or
 * synchronises); LBM_MEM_HOST: synchronising.  Errors (LBM_ERR_INVALID_ARG):
 * null pointers, bad mem flag, no state yet, planes outside the handle's
 * last axis. */
int lbm_get_planes(lbm_handle* h, int first, int count, void* buf, int mem);
int lbm_set_planes(lbm_handle* h, int first, int count, const void* buf, int mem);

/* Collide only planes [first, first + count) of the last axis in later steps
 * of the fused step form (a slab's owned planes; count = 0 restores the whole
 * axis).  The moment and force stages still read the two planes beyond each
 * end, which must hold valid populations; planes outside the range keep stale
 * values apart from the pushes of the range's edge planes.  The three-launch
 * form collides every plane regardless; a slab's exchange overwrites the
 * planes outside the range either way.  Errors (LBM_ERR_INVALID_ARG): null
 * handle, range outside the last axis. */
int lbm_set_step_planes(lbm_handle* h, int first, int count);

/* One step of the fused form in pieces, so that a slab can step the planes
 * next to its cuts first and swap them with its neighbours while its interior
 * steps (the step of Sec. 2-4 is the same per node whatever the order in
 * which planes are collided: every plane reads the step's input and writes
 * its own pushes).  lbm_step_begin collides planes [first, first + count) of
 * the last axis, asynchronously on the handle's stream.  The first call of a
 * step opens it: from then on the step's output is the handle's current
 * state, so lbm_get_planes / lbm_set_planes / lbm_get_crossing /
 * lbm_set_crossing act on planes the launches so far have written, and the
 * step count (the FP16 rounding seed) has advanced.  Later calls add ranges to
 * the same step; the ranges of one step must not overlap.  lbm_step_end
 * closes the step.  A range stepped this way writes exactly what lbm_step
 * writes for those planes, so ranges that cover [0, nm) (or the range of
 * lbm_set_step_planes) reproduce lbm_step bit for bit.  While a step is open,
 * lbm_step, lbm_profile_step, lbm_init, lbm_set_state, lbm_get_state and
 * lbm_moments_f refuse (LBM_ERR_INVALID_ARG; the last two use the idle
 * population buffer, which is the open step's input).  Errors (LBM_ERR_INVALID_ARG): null handle, no state
 * yet, a range outside the last axis, the three-launch step form; lbm_step_end
 * with no open step. */
int lbm_step_begin(lbm_handle* h, int first, int count);
int lbm_step_end(lbm_handle* h);

/* The populations that cross a cut of the last axis, for the first exchange
 * round between processes: bytes of one plane's pairs (N_k, g_k) for the
 * directions whose velocity component along the last axis is +1 (the same
 * count for -1): 5 directions for D3Q19, 3 for D2Q9. */
size_t lbm_crossing_bytes(const lbm_handle* h);

/* Copy those pairs of plane `plane` (sign +1 or -1 selects the directions)
 * out of / into buf, laid out as one row of the plane's nodes per direction
 * in increasing k, storage format.  mem as for lbm_get_planes (device:
 * asynchronous on the handle's stream; host: synchronising).  With walls on
 * x (or on y of D3Q19), lbm_set_crossing leaves alone the wall column (row)
 * of each direction whose velocity points away from that wall: no node
 * pushes those populations across the cut (they would come from beyond the
 * wall); the receiving node's own bounce-back wrote them in its step.  With
 * such walls and a host buffer, or a device buffer not aligned to a pair, it
 * stages the rows in the handle's host-transfer buffer (allocated on first
 * use, as by lbm_moments with host pointers).  Errors
 * (LBM_ERR_INVALID_ARG): null pointers, bad mem flag, sign not +1 / -1, no
 * state yet, plane outside the last axis. */
int lbm_get_crossing(lbm_handle* h, int plane, int sign, void* buf, int mem);
int lbm_set_crossing(lbm_handle* h, int plane, int sign, const void* buf, int mem);

/* The paper has no counterpart to this call: it is library plumbing for
 * callers that cannot allocate device memory, either because all their
 * device memory belongs to another framework's pool or because an allocation
 * would synchronise the device and stall their other work.
 *
 * Computes the FP64 Kahan sums of lbm_diagnostics (sums[0] mass, sums[1..3]
 * momentum x, y, z, sums[4] internal energy) of a population buffer the
 * caller owns, without allocating: `populations` is device memory holding
 * the 2Q planes of a state in `storage` format, laid out as lbm_get_state
 * writes them after its 16-byte header (N_0..N_{Q-1}, g_0..g_{Q-1}, each
 * nx*ny*nz values, x fastest); rho_ref and E_ref are the FP16 shifts (used
 * only with LBM_STORE_FP16).  `sums` is device memory for 5 doubles, written
 * asynchronously on `stream` (NULL: default stream); the caller synchronises.
 *
 * Scratch: a fixed 40,960-byte array in the library image, held by every
 * device that loads the library until exit.  The first call on a device
 * looks up that array's device address (with the device current) and should
 * come before any stream capture; the address is kept for the life of the
 * process, so do not use the call on a device after cudaDeviceReset.  Calls
 * share the array, so calls whose kernels overlap on the GPU race; calls
 * ordered on one stream do not (each overwrites every partial it reads).
 * Rejects null pointers, unknown lattice or storage, and sizes of 2^31 nodes
 * or more, the largest domain lbm_create accepts (LBM_ERR_INVALID_ARG);
 * launch failures give LBM_ERR_CUDA. */
int lbm_conservation_sums_noalloc(int lattice, int storage, int nx, int ny, int nz, double rho_ref,
                                  double E_ref, const void* populations, double* sums, void* stream);

/* Test hook, not for production runs.  From the next lbm_step on, the first
 * CTA of every fused step of this handle withholds the hand-off of plane
 * `plane` (index along the last lattice axis), so that its consumers' bounded
 * wait runs out and the next synchronising call reports LBM_ERR_TIMEOUT;
 * the steps run a separately compiled instance of the producer-load kernel
 * that carries the hook (the kernels of ordinary steps have no trace of it).
 * plane < 0 switches the hook off.  Errors: LBM_ERR_INVALID_ARG for a null
 * handle. */
int lbm_test_drop_handoff(lbm_handle* h, int plane);

/* Message of the last error on this thread ("" if none). */
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
