/*
 * cuba.h — C ABI of the GB300 test-particle transport library.
 *
 * One time step of the test-particle solution of the relativistic Boltzmann
 * equation for massless particles (arXiv:1208.0961, "CuBA - a CUDA
 * implementation of BAMPS"):
 *   A1 free streaming x -> x + (p_x / E) dt                 (Sec. 2, Eq. 2)
 *   A2 elastic reflection at the six box walls               (Sec. 2)
 *   A3 cell key of the new position                          (Sec. 2, PIC cells)
 *   A4 stable counting sort of the particles by cell         (Sec. 2, PIC cells)
 *   A5 every pair i < j of a cell is accepted iff u_ij < P22,
 *      P22 = v_rel sigma / N_test dt / V_cell,
 *      v_rel = s / (2 E_i E_j)                               (Sec. 2, Eq. 3)
 *   A6 conflicts: accepted pairs of a cell are executed greedily in
 *      lexicographic (i, j) order; a particle collides at most once per step
 *      (the paper is silent; this is the library's reading)
 *   A7 executed pairs are boosted to their centre-of-mass frame, given an
 *      isotropic direction and boosted back                  (Sec. 2)
 *   A8 per-cell T^00, T^0x, counts and global totals in FP64 (Sec. 5, Figs. 2-3)
 *
 * Units: fm, fm/c (c = 1), GeV; cross sections in fm^2 (1 mb = 0.1 fm^2).
 *
 * Random numbers are Philox4x32-10 keyed by the simulation seed with counters
 * (step, cell, i, j): a step is a pure function of the state, the seed and the
 * step index, independent of launch shape, batch composition and GPU.
 *
 * Conventions for every entry point:
 *  - Return value 0 on success or a negative CUBA_ERR_* code; the message of
 *    the last failure on the calling thread is cuba_last_error().
 *  - Pointers named "device" must be CUDA device (or managed) memory; pointers
 *    named "host or device" may be either (the copy direction is inferred by
 *    unified addressing); "host" means ordinary or pinned host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls marked "async" only enqueue work; errors raised by the
 *    kernels themselves (list overflow) surface in the next synchronous call.
 *  - The library owns all simulation state; callers own every buffer they
 *    pass in.  Objects are not thread-safe: one thread at a time per object.
 *  - The state layout is SoA, six arrays of n elements in this order:
 *    x, y, z, px, py, pz; element type double (CUBA_FP64) or float
 *    (CUBA_FP32), particles sorted by cell (stable within a cell).
 */
#ifndef CUBA_H
#define CUBA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CUBA_OK 0
#define CUBA_ERR_INVALID (-1)  /* bad argument or parameter */
#define CUBA_ERR_OOM (-2)      /* device or host allocation failed */
#define CUBA_ERR_CUDA (-3)     /* a CUDA runtime call failed */
#define CUBA_ERR_OVERFLOW (-4) /* accepted-pair list of a step overflowed; that
                                  step's collisions are incomplete */
#define CUBA_ERR_P22 (-5)      /* parameters give P22 > 1 (2 C > 1) */
#define CUBA_ERR_CAPACITY (-6) /* more particles or cells than reserved */

#define CUBA_FP32 0
#define CUBA_FP64 1

/* Parameters of one simulation (Sec. 2 and Sec. 5). */
typedef struct cuba_params {
    double L[3];          /* box edge lengths, fm; walls at 0 and L[a] */
    int32_t n_cells[3];   /* cells per axis; V_cell = (L0/n0)(L1/n1)(L2/n2) */
    double dt;            /* time step, fm/c; must be below every cell edge
                             (Sec. 5: dt < dx) so a particle crosses at most
                             one cell face per axis per step */
    double sigma_fm2;     /* total isotropic cross section, fm^2 (>= 0) */
    double n_test;        /* test particles per physical particle (> 0);
                             P22 is divided by it (Sec. 2) */
    int32_t precision;    /* CUBA_FP32 or CUBA_FP64 state and arithmetic */
    uint64_t seed;        /* Philox key of this simulation */
    double gamma_fp64;    /* CUBA_FP32 only: CM boosts with Lorentz factor
                             above this run in FP64 (<= 0: library default) */
    int32_t acceptance;   /* CUBA_ACCEPT_ALL_PAIRS (0): every pair i < j of a
                             cell draws its own uniform and is accepted iff
                             u < P22 (Sec. 2, Eq. 3), the paper's test.
                             CUBA_ACCEPT_SKIP (1): skip-ahead sampling of the
                             same distribution — candidates along each row
                             with geometric gaps at rate P_max = 2.0001 C,
                             each kept with probability P22 / P_max (no
                             counterpart in the paper; needs 2.0001 C < 1).
                             Each pair is accepted with probability P22
                             independently in both modes; the realisations
                             differ. */
    double kappa;         /* > 0: adaptive time step (no counterpart in the
                             paper, which names a variable dt as future work,
                             Sec. 6): each step takes
                             dt = ((kappa N_test) V_cell) / (sigma (n_max - 1))
                             with n_max the most populated cell at the start
                             of the step, so that its particles expect kappa
                             collisions; capped by dt (the field above), which
                             is used as is without collisions.  0: fixed dt.
                             At most 1/2 (keeps 2 C <= 1). */
    double mass;          /* particle mass m, GeV (0: the paper's massless
                             gluons).  E = sqrt(|p|^2 + m^2) everywhere; v_rel
                             is the Moller velocity sqrt((p_i.p_j)^2 - m^4) /
                             (E_i E_j); thermal sampling follows the Juttner
                             spectrum.  No counterpart in the paper. */
    double mu;            /* > 0: screened forward-peaked scattering,
                             dsigma/dt ~ 1/(t - mu^2)^2 in the CM frame (mu in
                             GeV); 0: isotropic (the paper's case).  The total
                             cross section, and so P22, is sigma either way.
                             With CUBA_FP32 these collisions run in FP64 (the
                             incoming CM direction cancels in FP32). */
} cuba_params;

#define CUBA_ACCEPT_ALL_PAIRS 0
#define CUBA_ACCEPT_SKIP 1

/* Thermal region for cuba_init_thermal: an axis-aligned box at temperature T. */
typedef struct cuba_region {
    double lo[3], hi[3]; /* fm, inside [0, L] */
    double T;            /* GeV (> 0) */
} cuba_region;

/* Counters accumulated over all steps of a simulation. */
typedef struct cuba_counters {
    int64_t steps;        /* steps taken */
    int64_t pair_tests;   /* pairs i < j tested (A5) */
    int64_t accepted;     /* pairs with u < P22 (A5) */
    int64_t executed;     /* pairs that collided (A6) */
    int64_t reflections;  /* wall reflections, one per axis crossing (A2) */
    int64_t fp64_boosts;  /* CUBA_FP32: collisions done in FP64 (A7) */
    int64_t overflow;     /* accepted pairs dropped for lack of list space */
    int64_t candidates;   /* CUBA_ACCEPT_SKIP: candidate pairs drawn (P22
                             evaluated); 0 in the all-pairs mode */
} cuba_counters;

typedef struct cuba_sim cuba_sim;

/*
 * Create a simulation with room for up to max_particles particles.  Checks
 * the parameters: L > 0, n_cells >= 1, 0 < dt < every cell edge, sigma >= 0,
 * n_test > 0, precision valid, 2 C <= 1 with C = sigma dt / (n_test V_cell)
 * (P22 <= 2 C since v_rel <= 2).  Allocates the device state on the current
 * device.  On success *out owns it until cuba_destroy.
 */
int cuba_create(const cuba_params* params, int64_t max_particles, cuba_sim** out);

/*
 * Device memory supplied by the caller.  Every device buffer of a simulation
 * or batch created with an allocator — state, sort and cell tables, the
 * accepted-pair list (allocated and grown by the synchronous calls that load
 * or sample a state), scratch, temporaries of synchronous calls — comes from
 * alloc and goes back through free; for that object the library calls
 * neither cudaMalloc nor cudaFree.  This lets a caching allocator (PyTorch's,
 * a memory pool) own the HBM that a server budgets.
 *   alloc(bytes, ctx): device memory of the current device, aligned to at
 *     least 256 bytes, or NULL; NULL fails the calling entry point with
 *     CUBA_ERR_OOM and a misaligned block with CUBA_ERR_INVALID (after giving
 *     it back).  Called from creation and from synchronous entry points only.
 *   free(ptr, bytes, ctx): take back a block alloc returned; bytes is the
 *     size that was asked for.  The library synchronizes the device before
 *     it calls free, so no kernel still uses the block.
 * The struct is copied at creation; ctx must stay valid until the object is
 * destroyed, and both callbacks must be non-NULL (CUBA_ERR_INVALID).
 */
typedef struct cuba_allocator {
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free)(void* ptr, size_t bytes, void* ctx);
    void* ctx;
} cuba_allocator;

/* cuba_create with every device buffer taken from `allocator` (above). */
int cuba_create_with_allocator(const cuba_params* params, int64_t max_particles, const cuba_allocator* allocator,
                               cuba_sim** out);

/*
 * Device bytes a simulation with these parameters and max_particles asks
 * for: everything allocated at creation plus the smallest accepted-pair list
 * (2^20 entries of 8 bytes, allocated by the first state load).  The list
 * grows to four times the per-cell room of the loaded state when that is
 * larger; tracing adds 4 max_particles bytes.  -1 for invalid arguments.
 * Pure arithmetic: no CUDA call.
 */
int64_t cuba_sim_bytes(const cuba_params* params, int64_t max_particles);

/* Free everything a simulation owns (NULL is ignored). */
void cuba_destroy(cuba_sim* sim);

/*
 * Sample n massless particles from thermal Boltzmann distributions: region r
 * receives a share of n proportional to T_r^3 V_r (largest remainder); in
 * it, positions are uniform and E ~ E^2 exp(-E/T) with isotropic directions.
 * Particle g (generation order) draws Philox blocks (0xFFFFFFFF, g_lo, g_hi, 0)
 * and (…, 1).  The state is then sorted by cell and the step counter reset
 * to 0.  Synchronous.
 */
int cuba_init_thermal(cuba_sim* sim, int64_t n, const cuba_region* regions, int n_regions,
                      void* stream);

/* The 1D Riemann initial state of Sec. 5: left half of the box (x < L0/2) at
   T_left, right half at T_right.  Same as cuba_init_thermal with two regions. */
int cuba_init_riemann(cuba_sim* sim, int64_t n, double T_left, double T_right, void* stream);

/*
 * Hot-spot initial state (the 3D thermal box with a hot spot): local
 * temperature T(r) = T0 + dT exp(-|r - c|^2 / (2 width^2)) about the box
 * centre c, density proportional to T(r)^3 (positions by rejection against
 * (T(r)/(T0 + dT))^3, at most 64 tries per particle, then the last try is
 * kept), E ~ E^2 exp(-E/T(r)) with isotropic directions.  Particle g uses the
 * Philox blocks (0xFFFFFFFF, g, 0, 2 + k) for its tries and (…, 0), (…, 1)
 * for its momentum.  Sorted by cell afterwards, step counter reset to 0.
 * Synchronous.
 */
int cuba_init_hotspot(cuba_sim* sim, int64_t n, double T0, double dT, double width, void* stream);

/*
 * Load a state of n particles (SoA x, y, z, px, py, pz of the simulation's
 * element type, host or device memory, any order); the library sorts it by
 * cell, stably.  Positions must lie in [0, L].  Synchronous.
 */
int cuba_set_state(cuba_sim* sim, const void* soa, int64_t n, void* stream);

/* Copy the current (cell-sorted) state, 6 n elements, to host or device
   memory.  Synchronous. */
int cuba_get_state(cuba_sim* sim, void* soa_out, void* stream);

/* Number of particles and of cells. */
int cuba_sizes(const cuba_sim* sim, int64_t* n_particles, int64_t* n_cells);

/* Step counter: index of the next step (the first counter word of its random
   numbers).  set_step lets a resumed run continue its random sequence. */
int cuba_get_step(const cuba_sim* sim, uint32_t* step);
int cuba_set_step(cuba_sim* sim, uint32_t step);

/* Simulated time (FP64 sum of the steps' dt since the last init or
   set_state, fm/c) and the dt of the last step taken (the fixed dt before the
   first one).  Synchronous.  Either pointer may be NULL. */
int cuba_get_time(const cuba_sim* sim, double* time, double* last_dt);

/*
 * Advance n_steps time steps A1-A7.  Async on `stream`: the work is replayed
 * from a captured CUDA graph of one step.
 */
int cuba_step(cuba_sim* sim, int n_steps, void* stream);

/*
 * A8 observables of the current state, per cell c (key ix + nx (iy + ny iz)):
 * T00[c] = sum E / (n_test V_cell), T0x[c] = sum p_x / (n_test V_cell), both
 * summed in FP64, counts[c] = particles.  Caller-owned host or device buffers
 * of n_cells elements; any may be NULL.  Synchronous; reports kernel errors.
 */
int cuba_observables(cuba_sim* sim, double* T00, double* T0x, int32_t* counts, void* stream);

/* FP64 totals {E, Px, Py, Pz} (host array) and the particle count.
   Synchronous; reports kernel errors. */
int cuba_totals(cuba_sim* sim, double out[4], int64_t* n_particles, void* stream);

/* Counters since creation (host struct).  Synchronous; reports kernel errors. */
int cuba_stats(cuba_sim* sim, cuba_counters* out);

/*
 * Launch shape of the collision step (no counterpart in the paper, which uses
 * one thread per particle).  Cells with 2 <= n <= small_max particles take
 * the warp-per-cell path (one warp tests all pairs of a cell, one warp
 * resolves it); larger cells are split into 32-row items that persistent
 * warps take from a queue.  small_max in [0, 1024]; 0 sends every cell to the
 * item path.  Default 32.  Results do not depend on it.
 */
int cuba_set_small_max(cuba_sim* sim, int32_t small_max);
int cuba_get_small_max(const cuba_sim* sim, int32_t* small_max);

/*
 * Autotuner: time n_steps steps for each candidate small_max
 * {0, 16, 32, 64, 128, 256, 512, 1024}, each from the same saved copy of the
 * present state (the simulation does not advance), and keep the fastest.
 * *chosen (optional) receives it, ms_per_candidate (optional, host, 8
 * doubles) the device time per step of each candidate.  Synchronous;
 * allocates a temporary copy of the state.
 */
int cuba_autotune(cuba_sim* sim, int n_steps, int32_t* chosen, double* ms_per_candidate, void* stream);

/*
 * The whole launch shape of the collision step: small_max as above, and the
 * Philox blocks a lane draws per loop iteration in the warp-per-cell pair
 * kernel (small_blocks: 1 or 2, default 2) and in the 32-row item kernel
 * (tile_blocks: 2, 4 or 8, default 4).  Results do not depend on it.
 */
typedef struct cuba_launch_shape {
    int32_t small_max;
    int32_t small_blocks;
    int32_t tile_blocks;
} cuba_launch_shape;

int cuba_set_launch_shape(cuba_sim* sim, const cuba_launch_shape* shape);
int cuba_get_launch_shape(const cuba_sim* sim, cuba_launch_shape* shape);

/*
 * Autotuner of the whole shape, by coordinates: small_max over the eight
 * candidates of cuba_autotune, then small_blocks in {1, 2}, then tile_blocks
 * in {2, 4, 8}, each candidate timed over n_steps steps from the same saved
 * state (the simulation does not advance); the fastest value of each
 * coordinate is kept before the next.  *chosen (optional) receives the shape,
 * ms_per_candidate (optional, host, 13 doubles) the device time per step of
 * the eight small_max candidates, then small_blocks 1, 2, then tile_blocks
 * 2, 4, 8.  Synchronous; allocates a temporary copy of the state.
 */
int cuba_autotune_shape(cuba_sim* sim, int n_steps, cuba_launch_shape* chosen, double* ms_per_candidate,
                        void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* cuba_last_error(void);

/*
 * Parity support.  With tracing on, each step keeps: the cell key of every
 * particle after streaming (pre-sort order), the sort permutation (sorted
 * position -> pre-sort index), cell_start (n_cells + 1) and the accepted
 * pairs with their executed flags.  cuba_trace_get copies them to host
 * buffers (any may be NULL): pairs as (cell, i, j) triples in lexicographic
 * order, executed[k] = 1 if pair k collided.  At most `cap` pairs are
 * written; *n_pairs receives the total.  Synchronous.
 */
int cuba_trace_enable(cuba_sim* sim, int on);
int cuba_trace_get(cuba_sim* sim, uint32_t* keys, uint32_t* perm, uint32_t* cell_start,
                   uint32_t* pairs, uint8_t* executed, int64_t cap, int64_t* n_pairs);

/*
 * Advance n_steps steps like cuba_step, but launched kernel by kernel (no
 * graph) with CUDA events between the phases; phase_ms (host, 6 doubles)
 * receives the summed device time of each phase over the steps:
 * [0] stream/reflect/key with the first digit histogram (or, for arenas of
 * many small cells, the neighbour-move sort's counting pass), [1] the rest of
 * the sort (scans, radix passes or the neighbour offsets, the final pass that
 * re-streams each particle into its sorted slot, cell_start),
 * [2] per-cell preparation, [3] pair kernels (including the survivor
 * kernel), [4] conflicts + kinematics, [5] step counter.  Synchronous.  For
 * measurement.
 */
int cuba_step_profiled(cuba_sim* sim, int n_steps, double* phase_ms, void* stream);

/*
 * The FP32 path's collision kinematics (A7) on given momenta: pair k is
 * particles (2k, 2k+1) of cell 0 at step `step` (random direction from the
 * Philox block (step, 0, 2k, 0x80000000 | (2k+1)) under `key`), boosted in
 * FP32 unless its CM Lorentz factor exceeds gamma_fp64, then in FP64.
 * pin/pout: device, 6 floats per pair (p_i then p_j); used_fp64: device, one
 * int per pair.  Async.  For choosing and checking the FP64 threshold.
 */
int cuba_kinematics_fp32(const float* pin, int64_t npairs, uint64_t key, uint32_t step, double gamma_fp64,
                         float* pout, int32_t* used_fp64, void* stream);

/*
 * Philox4x32-10 of the library's device implementation for n counters
 * (4 words each) under one key, into out (4 words each).  ctr and out are
 * device pointers.  Async.  For verifying the generator.
 */
int cuba_philox(const uint32_t* ctr, int64_t n, uint64_t key, uint32_t* out, void* stream);

/* ------------------------------------------------------------------------ */
/* Batches: many independent simulations advanced by one launch sequence.    */
/* ------------------------------------------------------------------------ */
/*
 * A batch holds the state of many simulations (each with its own box, cells,
 * dt, sigma, N_test, seed and step counter) in one device arena; every
 * cuba_batch_step advances all resident simulations by the same number of
 * steps with one captured graph per step (stream/key, one sort of the whole
 * arena, one persistent pair-tile launch over all cells of all simulations,
 * resolve).  Results of a simulation do not depend on the other residents:
 * its random numbers are keyed by its own seed, step counter and local cell
 * and particle indices, and every per-cell operation is order independent.
 * This is the execution layer for ensembles and for serving (the paper runs
 * one simulation at a time).
 */
typedef struct cuba_batch cuba_batch;

typedef struct cuba_batch_config {
    int32_t precision;      /* CUBA_FP32 or CUBA_FP64 for all members */
    int32_t max_sims;       /* resident simulations at most */
    int64_t max_particles;  /* particles of all residents together */
    int64_t max_cells;      /* cells of all residents together */
} cuba_batch_config;

/* Allocate an empty batch on the current device. */
int cuba_batch_create(const cuba_batch_config* cfg, cuba_batch** out);
/* The same with every device buffer taken from `allocator` (see
   cuba_allocator). */
int cuba_batch_create_with_allocator(const cuba_batch_config* cfg, const cuba_allocator* allocator,
                                     cuba_batch** out);
void cuba_batch_destroy(cuba_batch* b);

/*
 * Admit a simulation: params as for cuba_create (precision must match the
 * batch), n particles sampled like cuba_init_thermal.  Fails with
 * CUBA_ERR_CAPACITY (nothing changes) if the batch lacks room.  *id receives
 * a handle valid until cuba_batch_remove.  Synchronous.
 */
int cuba_batch_add(cuba_batch* b, const cuba_params* params, int64_t n, const cuba_region* regions,
                   int n_regions, int32_t* id, void* stream);

/* Same with a given state (SoA x, y, z, px, py, pz of n particles, host or
   device memory, any order) instead of sampling.  Synchronous. */
int cuba_batch_add_state(cuba_batch* b, const cuba_params* params, const void* soa, int64_t n, int32_t* id,
                         void* stream);

/* Retire a simulation and compact the arena.  Synchronous. */
int cuba_batch_remove(cuba_batch* b, int32_t id);

/* Advance every resident simulation by n_steps.  Async on `stream`. */
int cuba_batch_step(cuba_batch* b, int n_steps, void* stream);

/* Per-member queries, as the single-simulation calls (synchronous). */
int cuba_batch_observables(cuba_batch* b, int32_t id, double* T00, double* T0x, int32_t* counts, void* stream);
int cuba_batch_totals(cuba_batch* b, int32_t id, double out[4], int64_t* n_particles, void* stream);
int cuba_batch_stats(cuba_batch* b, int32_t id, cuba_counters* out);
int cuba_batch_get_state(cuba_batch* b, int32_t id, void* soa_out, void* stream);
int cuba_batch_get_step(cuba_batch* b, int32_t id, uint32_t* step);
int cuba_batch_get_time(cuba_batch* b, int32_t id, double* time, double* last_dt);

/* Autotuner and launch shape of a batch, as cuba_autotune / cuba_set_small_max
   (all resident members are timed together; none advances). */
int cuba_batch_autotune(cuba_batch* b, int n_steps, int32_t* chosen, double* ms_per_candidate, void* stream);
int cuba_batch_set_small_max(cuba_batch* b, int32_t small_max);
int cuba_batch_set_launch_shape(cuba_batch* b, const cuba_launch_shape* shape);
int cuba_batch_get_launch_shape(cuba_batch* b, cuba_launch_shape* shape);
int cuba_batch_autotune_shape(cuba_batch* b, int n_steps, cuba_launch_shape* chosen, double* ms_per_candidate,
                              void* stream);

/* Occupancy: resident simulations, particles and cells in use. */
int cuba_batch_usage(const cuba_batch* b, int32_t* n_sims, int64_t* n_particles, int64_t* n_cells);

/* Device bytes a batch of this configuration asks for: everything allocated
   at creation plus the smallest accepted-pair list (2^20 entries of 8 bytes,
   allocated by the first admission).  The list grows, at admissions, to four
   times the per-cell room of the residents when that is larger (room of a
   cell of n particles: mu + 8 sqrt(mu) + 16 entries, mu = 2.0001 C n (n - 1)
   / 2); a server budgets that on top.  -1 for an invalid configuration.
   Pure arithmetic: no CUDA call. */
int64_t cuba_batch_bytes(const cuba_batch_config* cfg);

/*
 * Cell keys and stable sort of particle positions without allocating memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory themselves -- code running inside a region
 * that forbids allocation (a frame budget of a real-time loop, a memory pool
 * that must not grow, a caller that has no CUDA allocator of its own) -- and
 * still want the binning step (A3, A4) of the library.
 *
 * params: as for cuba_create (host struct; checked the same way).
 * xyz: device, SoA positions x[n], y[n], z[n] of the params' precision.
 * perm: device, n uint32 out: perm[k] = input index of the particle at sorted
 * position k (stable within a cell).  cell_start: device, n_cells + 1 uint32
 * out: first sorted position of each cell, cell_start[n_cells] = n.
 * Async on `stream`.
 *
 * No cudaMalloc, cudaFree or allocating library call is made.  All scratch
 * lives in one fixed device array inside the library, sized for
 * CUBA_NOALLOC_MAX_PARTICLES particles (about 4 MiB); every GPU that loads the
 * library holds it until the process exits.  n above the maximum fails with
 * CUBA_ERR_CAPACITY before any GPU work.  The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress), which may load the
 * library's device code; make that first call before any stream capture.
 * Every call on a device shares the one array: calls whose work overlaps on
 * the GPU (other streams, other host threads) race and corrupt each other's
 * results; serialise them.
 */
#define CUBA_NOALLOC_MAX_PARTICLES (1 << 18)
int cuba_bin_noalloc(const cuba_params* params, const void* xyz, int64_t n, uint32_t* perm,
                     uint32_t* cell_start, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CUBA_H */
