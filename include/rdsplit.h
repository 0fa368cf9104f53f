/*
 * rdsplit — operator-split stochastic reaction-diffusion on tetrahedral
 * meshes, on one NVIDIA GB300 (sm_103a).
 *
 * Method: Hepburn, Chen & De Schutter, "Accurate reaction-diffusion operator
 * splitting on tetrahedral meshes for parallel stochastic molecular
 * simulations" (arXiv:1512.03126), Algorithm 1.  In every period tau each
 * tetrahedron runs its own SSA reactions (Sec. II.C, Step 2), then each
 * species sends n = Binomial(N-bar, zeta) molecules (Eq. 3) to its face
 * neighbours multinomially (Sec. II.B), and the transfers are applied
 * synchronously.  Options: the paper's comparison transfer rules (Sec. II.C,
 * rdsplit_set_transfer_rule) and its outlier choice of tau (Sec. II.A,
 * rdsplit_set_zeta_outliers).  A triangle mesh passed with triangle areas as
 * volumes, edge lengths as face areas and the fourth neighbour -1 gives
 * surface diffusion (Sec. III.A).
 *
 * Conventions for every call:
 *   - Return value: 0 on success, else a negative RDSPLIT_E* code; the text
 *     of the last error on the calling thread is rdsplit_last_error().
 *   - Host arrays passed in are copied during the call; the caller keeps
 *     ownership.  Output arrays are caller-owned and must have the stated
 *     size.
 *   - Tet order: all arrays use the caller's (canonical) tet order; random
 *     streams are keyed by canonical tet ids, so results never depend on how
 *     the library stores or schedules tets.
 *   - Counts are int32 [n_tets][n_species], tet-major.
 *   - All device work of a handle is issued on its stream (default: the
 *     legacy default stream; see rdsplit_set_stream) and every call that
 *     returns host-visible results synchronises that stream.
 *   - A handle must not be used from two threads at once.
 */
#ifndef RDSPLIT_H
#define RDSPLIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RDSPLIT_OK 0
#define RDSPLIT_EINVAL (-1)    /* bad argument, malformed mesh or model */
#define RDSPLIT_ENOMEM (-2)    /* device allocation failed or budget exceeded */
#define RDSPLIT_ECUDA (-3)     /* a CUDA runtime call failed */
#define RDSPLIT_ETIMEOUT (-4)  /* reserved: no call returns it (the kernels wait
                                  only at hardware barriers, never on a flag) */
#define RDSPLIT_EOVERFLOW (-5) /* a count would exceed INT32_MAX, or a
                                  period would exceed the per-tet event cap */
#define RDSPLIT_ESTATE (-6)    /* call out of order (e.g. run before set_model) */

#define RDSPLIT_MAX_SPECIES 16
#define RDSPLIT_MAX_REACTIONS 32

typedef struct rdsplit_mesh* rdsplit_mesh_t;

/* Text of the last error raised on the calling thread ("" if none). */
const char* rdsplit_last_error(void);

/*
 * Create a mesh handle from the geometry of Sec. II.A: irregular tetrahedral
 * subvolumes with up to 4 face neighbours each.
 *   n_tets         number of tets, > 0
 *   adj            int32 [n_tets][4]; adj[t][f] = neighbour across face f, or
 *                  -1 (reflective boundary).  Must be symmetric: if
 *                  adj[t][f] = u then exactly one r has adj[u][r] = t.
 *   vol            float64 [n_tets], m^3, > 0
 *   face_area      float64 [n_tets][4], m^2, >= 0
 *   centroid_dist  float64 [n_tets][4], m, distance between the centroids of
 *                  t and adj[t][f]; > 0 where adj >= 0, ignored elsewhere
 *   flags          0 (RDSPLIT_REORDER_SFC needs the centroids: see
 *                  rdsplit_mesh_create_ex)
 *   out            receives the handle
 * The face coefficient g = A / (V dist) and the reverse-face table are
 * computed on the device; validation runs there too and a malformed mesh
 * returns RDSPLIT_EINVAL.
 */
int rdsplit_mesh_create(int32_t n_tets, const int32_t* adj, const double* vol,
                        const double* face_area, const double* centroid_dist,
                        int32_t flags, rdsplit_mesh_t* out);

/*
 * Same, with the tet centroids, so that the library can store the tets in
 * its own order.
 *   centroid       float64 [n_tets][3], m (finite), or NULL without a
 *                  reordering flag
 *   flags          0, or RDSPLIT_REORDER_SFC: store the tets along a Morton
 *                  (Z-order) curve of their centroids (the box of the
 *                  centroids cut into 2^21 steps per axis, ties by tet id),
 *                  so that the tets a warp handles together are neighbours
 *                  in space whatever the caller's numbering
 * The reordering is internal: every array the caller passes or reads stays
 * in the caller's (canonical) tet order, and random streams stay keyed by
 * canonical ids, so results do not depend on the flag.
 */
#define RDSPLIT_REORDER_SFC 1
int rdsplit_mesh_create_ex(int32_t n_tets, const int32_t* adj, const double* vol,
                           const double* face_area, const double* centroid_dist,
                           const double* centroid, int32_t flags, rdsplit_mesh_t* out);

/* The stored order: perm[i] (int32 [n_tets], host) = canonical id of the
 * i-th stored tet (the identity without a reordering). */
int rdsplit_get_order(rdsplit_mesh_t mesh, int32_t* perm);

/*
 * Attach a chemistry (Sec. III.C: species with diffusion constants,
 * mass-action reactions with rate constants) and compute the period
 * tau = tau_scale / max_{s,t}(D_s * sum_f g_tf)  (Algorithm 1, precompute;
 * tau_scale < 1 is the "reduce zeta everywhere" option of Sec. II.A).
 *   n_species      1..RDSPLIT_MAX_SPECIES
 *   D              float64 [n_species], m^2/s, >= 0
 *   n_reactions    0..RDSPLIT_MAX_REACTIONS
 *   lhs, rhs       int32 [n_reactions][n_species] reactant / product
 *                  stoichiometry, >= 0, total reactant order <= 2
 *   k              float64 [n_reactions]; s^-1 (first order), M^-1 s^-1
 *                  (second order), M s^-1 (zero order, scaled by the tet
 *                  volume)
 *   rxn_tet_mask   uint8 [n_reactions][n_tets] (0 = reaction off in that
 *                  tet) or NULL (everywhere)
 *   tau_scale      in (0, 1]
 * Resets counts to zero, time to 0 and the period index to 0.
 */
int rdsplit_set_model(rdsplit_mesh_t mesh, int32_t n_species, const double* D,
                      int32_t n_reactions, const int32_t* lhs, const int32_t* rhs,
                      const double* k, const uint8_t* rxn_tet_mask, double tau_scale);

/*
 * Outlier option for tau (Sec. II.A): take tau = tau_scale / d_(k+1), d_(j)
 * the j-th largest per-tet rate max_s D_s * sum_f g_tf, instead of the
 * largest; the k fastest tets then have tau * d > 1 and run with zeta
 * capped at 1 (every molecule there leaves each period), a small cost to
 * accuracy that raises tau for a mesh with a few tiny tets.  k = 0 restores
 * the default.  Needs a model; rdsplit_set_model resets k to 0.  Recomputes
 * tau and the face thresholds on the device (a rank selection over G).
 *   k    0 <= k < n_tets, else RDSPLIT_EINVAL
 */
int rdsplit_set_zeta_outliers(rdsplit_mesh_t mesh, int32_t k);

/*
 * Diagnostic (Fig. 1d): histogram of zeta_t = min(1, tau * D_max * G_t) over
 * the tets, for the fastest species.
 *   nbins     1 .. 2^20; bin b holds zeta in [b/nbins, (b+1)/nbins), and
 *             zeta = 1 falls in the last bin
 *   counts    int64 [nbins] (host), filled
 *   mean      mean zeta over the tets, or NULL (summed with atomics: the last
 *             bits may vary between calls)
 *   max_zeta  largest zeta, or NULL
 * With no diffusing species (tau infinite) every zeta is reported as 0.
 */
int rdsplit_zeta_histogram(rdsplit_mesh_t mesh, int32_t nbins, int64_t* counts, double* mean, double* max_zeta);

/*
 * Transfer rule: which count of a period the diffusion draw of Step 3.2 uses
 * (Sec. II.C; the comparison of Sec. III.B, Fig. 7).
 *   RDSPLIT_TRANSFER_MEAN  N-bar, the mean occupancy over the period (Eq. 3);
 *                          the method, and the default
 *   RDSPLIT_TRANSFER_END   N(tau_k), the count after the reaction phase:
 *                          first-order operator splitting
 *   RDSPLIT_TRANSFER_MID   N(tau_k / 2), the count at mid-period: the reading
 *                          of N that half-step (Strang) splitting amounts to
 * Without reactions the three give identical results.  The rule is kept
 * across rdsplit_set_model and travels with the handle into the batched
 * engine.  Returns RDSPLIT_EINVAL for another value.
 */
#define RDSPLIT_TRANSFER_MEAN 0
#define RDSPLIT_TRANSFER_END 1
#define RDSPLIT_TRANSFER_MID 2
int rdsplit_set_transfer_rule(rdsplit_mesh_t mesh, int32_t rule);

/* Set counts from host memory, int32 [n_tets][n_species], all >= 0. */
int rdsplit_set_counts(rdsplit_mesh_t mesh, const int32_t* counts);
/* Same from device memory (same layout), e.g. a torch CUDA tensor. */
int rdsplit_set_counts_device(rdsplit_mesh_t mesh, const int32_t* d_counts);

/*
 * Advance from the current time t to t_end with Algorithm 1: periods of
 * length tau, the last one shortened to end on t_end (Step 1).  `seed` keys
 * every random draw together with the global period index, so that
 * run(t1) followed by run(t2) equals run(t2) whenever t1 falls on a period
 * boundary.  t_end <= t is a no-op.
 */
int rdsplit_run(rdsplit_mesh_t mesh, double t_end, uint64_t seed);

/* Advance exactly n_periods full periods of length tau (no alignment). */
int rdsplit_run_periods(rdsplit_mesh_t mesh, int64_t n_periods, uint64_t seed);

/* Copy counts to host memory, int32 [n_tets][n_species]. */
int rdsplit_get_counts(rdsplit_mesh_t mesh, int32_t* out);
/* Same into device memory. */
int rdsplit_get_counts_device(rdsplit_mesh_t mesh, int32_t* d_out);

/* Current time (s) and global period index. */
int rdsplit_get_time(rdsplit_mesh_t mesh, double* t, int64_t* period);
/* Set the current time and period index (checkpoint restore). */
int rdsplit_set_time(rdsplit_mesh_t mesh, double t, int64_t period);
/* The period tau (s) of the attached model; +inf if no species diffuses. */
int rdsplit_get_tau(rdsplit_mesh_t mesh, double* tau);
/* Number of tets / species of the handle. */
int rdsplit_get_shape(rdsplit_mesh_t mesh, int32_t* n_tets, int32_t* n_species);

/*
 * Kernel form of the period (Algorithm 1, Steps 2-3), a tuning choice with no
 * effect on results (every draw is keyed by tet and period):
 *   mode 1  one pass: gather, reactions and draws of each tet in one kernel
 *   mode 2  two passes: a light pass runs the tets that need neither the
 *           reaction phase nor the double-precision binomial (compiled
 *           without those samplers, so it keeps more warps per SM) and
 *           defers the others to a slow pass with the full step
 *   mode 0  automatic (default): one pass
 *   block   threads per block of the period kernel (of the light pass in
 *           mode 2): a multiple of 32 in 32..256, or 0 (default) for a size
 *           chosen from the mesh (smaller blocks for small meshes, so that
 *           their tets spread over all SMs)
 * rdsplit_get_period_kernel reports whether runs use two passes and the
 * block size they use.
 */
int rdsplit_set_period_kernel(rdsplit_mesh_t mesh, int32_t mode, int32_t block);
int rdsplit_get_period_kernel(rdsplit_mesh_t mesh, int32_t* two_passes, int32_t* block);

/*
 * Domain decomposition (Sec. III.D: each process advances its own tets to
 * tau, buffers the changes for tets of other processes, and the buffers are
 * exchanged and applied before the next period).  Each rank holds a handle
 * of the whole mesh and advances only its range of tets; the molecules its
 * tets send across cut faces land in inbox slots of tets it does not own,
 * which the rank exports and the owner imports before its next period.
 * Every draw is keyed by canonical tet ids, so the ranks together give the
 * single-process result bit for bit.
 *   rdsplit_partition_set    own tets [t0, t1) (not on a reordered mesh)
 *   rdsplit_partition_step   one period of Algorithm 1 for the own tets,
 *                            towards t_end exactly as rdsplit_run would take
 *                            it (the last period shortened); the first step
 *                            after set/end starts from the handle's counts;
 *                            *more = 1 while t < t_end.  No period is run
 *                            once t >= t_end.
 *   rdsplit_inbox_export     after a step: d_buf (device, int32 [n][S]) =
 *                            the molecules sent into inbox slots d_slots
 *                            (device, int32 [n]; slot 4 u + r is face r of
 *                            tet u) by this rank's tets
 *   rdsplit_inbox_import     after a step, before the next: writes d_buf
 *                            into the own tets' slots d_slots (what another
 *                            rank's tets sent them)
 *   rdsplit_partition_end    applies the last period's transfers to the own
 *                            tets; their counts then read as after
 *                            rdsplit_run (other tets' counts are not kept)
 * The slot lists are the caller's: for ranks owning [a0, a1) and [b0, b1),
 * the slots 4 u + r with u in [b0, b1) and adj[u][r] in [a0, a1), in
 * increasing order, are exported by the first and imported by the second.
 * Export and import synchronise the handle's stream before returning.
 */
int rdsplit_partition_set(rdsplit_mesh_t mesh, int32_t t0, int32_t t1);
int rdsplit_partition_step(rdsplit_mesh_t mesh, double t_end, uint64_t seed, int32_t* more);
int rdsplit_inbox_export(rdsplit_mesh_t mesh, const int32_t* d_slots, int32_t n, int32_t* d_buf);
int rdsplit_inbox_import(rdsplit_mesh_t mesh, const int32_t* d_slots, int32_t n, const int32_t* d_buf);
int rdsplit_partition_end(rdsplit_mesh_t mesh);

/* Issue all of the handle's device work on `stream` (a cudaStream_t). */
int rdsplit_set_stream(rdsplit_mesh_t mesh, void* stream);

/* Release the handle and its device memory. */
int rdsplit_mesh_destroy(rdsplit_mesh_t mesh);

/*
 * Device memory provider for all later allocations (e.g. PyTorch's caching
 * allocator).  alloc(bytes, ctx) returns a device pointer or NULL; free(ptr,
 * ctx) releases it.  NULL functions restore cudaMalloc / cudaFree.  Must not
 * be changed while handles allocated through the previous provider exist.
 */
typedef void* (*rdsplit_alloc_fn)(size_t bytes, void* ctx);
typedef void (*rdsplit_free_fn)(void* ptr, void* ctx);
int rdsplit_set_allocator(rdsplit_alloc_fn alloc, rdsplit_free_fn free_fn, void* ctx);

/* Number of kernels the library has launched on this process so far. */
int64_t rdsplit_kernel_launches(void);

/*
 * Profiling hook (tracing, no counterpart in the paper): when stride > 0,
 * every stride-th launch of the period kernel is bracketed by CUDA events on
 * the handle's stream and its device duration accumulated; stride = 0 turns
 * sampling off.  rdsplit_get_timing returns the summed milliseconds and the
 * number of sampled launches since the last rdsplit_set_timing call.
 */
int rdsplit_set_timing(rdsplit_mesh_t mesh, int32_t stride);
int rdsplit_get_timing(rdsplit_mesh_t mesh, double* total_ms, int64_t* n_sampled);

/*
 * Batched engine: many independent simulations advanced by one persistent
 * kernel in which each thread-block cluster (1, 2, 4 or 8 CTAs, see
 * rdsplit_engine_set_concurrency) takes one simulation from a queue
 * (largest first) and runs its periods itself, touching only tets that hold
 * molecules (or have a zero-order reaction switched on).  Realisations in
 * parallel are the embarrassingly parallel use of Sec. I; each simulation's
 * counts are exactly those rdsplit_run would give it alone (its random
 * streams are keyed by its own seed, period index and canonical tet ids),
 * whatever else runs beside it.
 *
 * rdsplit_engine_create: max_slots simultaneous simulations; max_active_tets
 *   bounds the sum of n_tets over simulations in the engine (admission limit).
 *   The first engine created on a device launches every engine kernel once
 *   with no work, on the legacy default stream, and waits for them (so that
 *   the concurrent group launches of a step never wait on a first launch);
 *   create it before any stream capture.
 * rdsplit_engine_add: a mesh handle with its model and counts joins; it will
 *   run from its current time to t_end with `seed` (as rdsplit_run would).
 *   RDSPLIT_ENOMEM if no slot or capacity is free.  The handle must not be
 *   used otherwise until it has finished.
 * rdsplit_engine_step: advance every active simulation by up to n_steps
 *   periods in one launch (a time slice); synchronises the engine's stream.
 *   Finished handles hold their final counts, time and period index.
 *   Between calls, simulations may be added (continuous batching).
 * rdsplit_engine_poll: slot ids of simulations finished since the last poll.
 * rdsplit_engine_active: number of active simulations and their total tets.
 * rdsplit_ensemble_run: convenience — run n handles to t_end[i] with
 *   seeds[i] in one engine (the batched ensemble, one launch).
 * All device work is issued on the engine's stream (rdsplit_engine_set_stream;
 * default: the legacy default stream); the meshes' own work must not overlap
 * it.
 */
typedef struct rdsplit_engine* rdsplit_engine_t;
int rdsplit_engine_create(int32_t max_slots, int64_t max_active_tets, rdsplit_engine_t* out);
int rdsplit_engine_set_stream(rdsplit_engine_t engine, void* stream);
int rdsplit_engine_add(rdsplit_engine_t engine, rdsplit_mesh_t mesh, double t_end, uint64_t seed,
                       int32_t* slot_out);
int rdsplit_engine_step(rdsplit_engine_t engine, int64_t n_steps);
int rdsplit_engine_poll(rdsplit_engine_t engine, int32_t* slots, int32_t max, int32_t* n_out);
int rdsplit_engine_active(rdsplit_engine_t engine, int32_t* n_slots, int64_t* n_tets);
int rdsplit_engine_destroy(rdsplit_engine_t engine);
/* Scheduling: `in_flight` simulations are processed at once (0 = as many
 * clusters as fit on the GPU at once; never more than that), each by a
 * thread-block cluster of `cluster` CTAs (1, 2, 4 or 8; default 2) whose
 * warps share its tets and meet at a cluster barrier every period.  More
 * CTAs per simulation shorten the longest simulations (large meshes with
 * many molecules), fewer serve more simulations at once.  A step's
 * simulations are launched in groups by species count and reactions, the
 * groups running concurrently with the in-flight clusters shared by work.
 * Fewer in flight keeps their working sets in L2.  RDSPLIT_EINVAL for any
 * other cluster size or a negative in_flight. */
int rdsplit_engine_set_concurrency(rdsplit_engine_t engine, int32_t in_flight, int32_t cluster);
/* Slices of equal cost: with max_tet_periods > 0, rdsplit_engine_step
 * advances a simulation of T tets by min(n_steps, max(1, max_tet_periods /
 * T)) periods, so that the largest simulations of a mix do not hold a
 * launch while the clusters that ran the small ones idle (continuous
 * batching).  0 (default) advances every simulation by n_steps.  Results
 * do not depend on the slicing. */
int rdsplit_engine_set_slice_work(rdsplit_engine_t engine, int64_t max_tet_periods);
/* Profiling: time every engine launch with CUDA events (on != 0), and read
 * the periods advanced (maximum per step call, summed), the (simulation, tet)
 * entries processed, and the summed milliseconds / number of timed launches. */
int rdsplit_engine_set_timing(rdsplit_engine_t engine, int32_t on);
int rdsplit_engine_stats(rdsplit_engine_t engine, int64_t* steps, int64_t* processed,
                         double* timing_ms, int64_t* timing_n);
/* Profiling: while timing is on, each launch records for every simulation it
 * runs the device clock (%globaltimer, ns) when its cluster takes it and when
 * it finishes its slice, and the (simulation, tet) entries it processed.
 * Copies int64 [n][3] (start, end, entries) for slots 0 .. n-1, n =
 * min(max_slots, engine slots); a slot not run since timing was switched on
 * holds what it held before (0 initially). */
int rdsplit_engine_slot_times(rdsplit_engine_t engine, int64_t* out, int32_t max_slots);
/* The schedule of the last launch: simulations in flight (clusters
 * launched), CTAs per cluster, and the number of clusters the occupancy
 * query says fit on the GPU at once (the default in-flight count). */
int rdsplit_engine_schedule(rdsplit_engine_t engine, int32_t* in_flight, int32_t* cluster, int32_t* max_active);
int rdsplit_ensemble_run(int32_t n, const rdsplit_mesh_t* meshes, const double* t_end,
                         const uint64_t* seeds);

/*
 * Allocation-free run.  The paper has no counterpart: this is a deployment
 * variant of rdsplit_run.  Some callers cannot call cudaMalloc: code running
 * inside a host application that owns all device memory (a plugin with a
 * fixed memory budget), or a real-time loop that must not stall on the
 * device synchronisation an allocation can cause.  This entry point performs
 * no device allocation or free of any kind: every intermediate array lives in
 * one static device array of RDSPLIT_STATIC_SCRATCH_BYTES that the library
 * reserves on each GPU that loads it, until the process exits.
 *
 * It runs the same period loop and kernels as rdsplit_run, with the same
 * results, on caller-owned memory:
 *   d_adj, d_vol, d_face_area, d_centroid_dist   the mesh, in DEVICE memory,
 *                 same layout and rules as rdsplit_mesh_create
 *   n_species, D, n_reactions, lhs, rhs, k      the model, in HOST memory,
 *                 same rules as rdsplit_set_model
 *   d_rxn_tet_mask   DEVICE uint8 [n_reactions][n_tets] or NULL
 *   d_counts      DEVICE int32 [n_tets][n_species]; read at the start,
 *                 overwritten with the counts at the end
 *   t, period     HOST in/out: current time and global period index
 *   t_end, seed   as for rdsplit_run
 *   stream        cudaStream_t for all work (NULL: legacy default stream);
 *                 the call synchronises it before returning
 * Scratch needed: rdsplit_static_scratch_bytes(n_tets, n_species, masked);
 * larger problems are rejected with RDSPLIT_EINVAL and a message giving
 * both sizes.
 * The first call on each device looks up the array's device address (with
 * that device current) and caches it; make that first call before any
 * stream capture.  All calls share the one array, which keeps the last
 * call's contents (the call clears what must start at zero): calls whose
 * device work overlaps, on any streams or threads, race on it and must be
 * serialised by the caller.
 */
#define RDSPLIT_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
size_t rdsplit_static_scratch_bytes(int32_t n_tets, int32_t n_species, int32_t masked);
int rdsplit_run_static(int32_t n_tets, const int32_t* d_adj, const double* d_vol,
                       const double* d_face_area, const double* d_centroid_dist,
                       int32_t n_species, const double* D, int32_t n_reactions,
                       const int32_t* lhs, const int32_t* rhs, const double* k,
                       const uint8_t* d_rxn_tet_mask, double tau_scale, int32_t* d_counts,
                       double* t, int64_t* period, double t_end, uint64_t seed,
                       void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RDSPLIT_H */
