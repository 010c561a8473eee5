/*
 * heat.h -- C ABI of the GB300 periodic 1D heat-stencil library (libheat.so).
 *
 * The operation (arXiv 2307.01117, Section 2 "Model problem"):
 *   Eq. 1  u_t = alpha u_xx on a loop of length L with periodic boundary
 *          u(t, x) = u(t, L + x);
 *   Eq. 2  forward Euler on N grid points x_i = i h with second-order central
 *          differences:  u'(x_i) = u(x_i) + r * ((u(x_{i-1}) - 2 u(x_i)) + u(x_{i+1})),
 *          r = k * dt / dx^2  (k = alpha, dx = h; the printed "2h" denominator is
 *          read as h^2, the value second-order differencing gives);
 *   Section 2, parallel algorithm: the ring is split into np segments of nx
 *          points; each segment is advanced by its own worker and ghost values
 *          cross between neighbouring segments through single-producer
 *          single-consumer queues.
 *
 * All arithmetic runs in the library's CUDA kernels (sm_103a).  Conventions for
 * every call:
 *   - Return value: HEAT_OK (0) or a negative heat_status code; heat_strerror()
 *     names it.  A NULL context argument returns HEAT_EINVAL.
 *   - Ownership: the context owns all device memory it allocates and frees it
 *     in heat_destroy().  Pointers passed in are borrowed for the duration of
 *     the call only.
 *   - Layout: state arrays are in global ring order g = p*nx + j (partition p,
 *     local index j), contiguous, N = np*nx elements.
 *   - Streams: work is queued on the context's stream (its own non-blocking
 *     stream unless heat_set_stream() names another).  heat_run() is
 *     asynchronous; errors that arise on the device (a bounded wait that ran
 *     out) are reported by the next synchronising call (heat_sync, heat_get,
 *     heat_sum, heat_get_device).
 *   - A context is not thread-safe: one host thread at a time.
 *
 * Citations: the entries that carry the operation (heat_create, heat_set,
 * heat_run, heat_get and their batch counterparts) implement Section 2 as cited
 * on each.  The entries that select kernels, tune, observe or test the library
 * (forms, layouts, graphs, segments, wait limits, fault hooks, info, the
 * batch runtime's arena and scheduler, the allocation-free stepper) have no
 * counterpart in the paper and say what they do instead.
 */
#ifndef HEAT_H
#define HEAT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct heat_ctx heat_ctx; /* opaque, library-owned */

/* Storage/arithmetic type of the ring state. */
typedef enum {
  HEAT_F64 = 0,  /* binary64 state; Eq. 2 in binary64 */
  HEAT_F32C = 1  /* binary32 state; update in binary32 with a TwoSum-compensated
                    correction carried within each temporal block (the paper
                    has no reduced-precision form; this is the library's) */
} heat_dtype;

typedef enum {
  HEAT_OK = 0,
  HEAT_EINVAL = -1,   /* bad argument (sizes, non-finite or zero coefficients, NULL) */
  HEAT_ENOMEM = -2,   /* device allocation failed */
  HEAT_ECUDA = -3,    /* a CUDA runtime call failed (launch, copy, sync) */
  HEAT_ETIMEOUT = -4, /* a bounded device wait on a neighbour's ghost ran out */
  HEAT_ESTATE = -5,   /* call not valid in the context's state */
  HEAT_ENOTSUP = -6   /* combination not supported (e.g. form for this dtype) */
} heat_status;

/* Kernel form used by heat_run().  All forms give bitwise the same result for
 * HEAT_F64 with HEAT_ARITH_EXACT (the segmented algorithm of Section 2 computes
 * every point with the same operation on the same operands as the unsegmented
 * ring). */
typedef enum {
  HEAT_FORM_PLAIN = 0,   /* one global step per launch; ghost exchange implicit
                            through the launch boundary (Section 3.1's
                            synchronous, unsegmented variant) */
  HEAT_FORM_PERSIST = 1, /* one persistent launch; each CTA owns a segment and
                            swaps ghost values with its neighbours through
                            device-memory flag queues (Section 2's SPSC queues).
                            Depth T: each message carries T edge values and the
                            segment advances T steps per message (register-
                            resident warp tiles, binary64 split between the
                            FP64 unit and the integer pipes as in the
                            temporal-blocking forms); T = 1: one value and one
                            step per message */
  HEAT_FORM_TBLOCK = 2,  /* temporal blocking: T steps per register-resident tile */
  HEAT_FORM_AUTO = 3,    /* library picks (measured fastest for each range):
                            HEAT_FORM_CLUSTER for every ring the cluster form
                            takes, HEAT_FORM_PERSIST_TB for binary64 rings under
                            the exact reading from 2^18 to 2^26 points,
                            HEAT_FORM_TBLOCK otherwise */
  HEAT_FORM_CLUSTER = 4, /* small rings (up to 16 x 4 windows of output, about
                            31000 binary64 points at T = 8): one thread-block
                            cluster of up to 16 CTAs runs all nt steps in one
                            launch; each CTA keeps its segment in shared memory
                            and reads its neighbours' T-point halos through
                            distributed shared memory, one cluster barrier per
                            block of T steps */
  HEAT_FORM_PERSIST_TB = 5 /* persistent temporal blocking: one launch for all
                            nt steps; the ring is cut into warp-sized tiles that
                            advance T steps at a time, each waiting (acquire/
                            release completion counters, bounded) until it and
                            its two neighbours finished the previous block --
                            the segmented algorithm of Section 2 with T-wide
                            ghost zones, no launch boundary between blocks */
} heat_form;

/* Rounding reading of Eq. 2 for HEAT_F64 (the paper states no order). */
typedef enum {
  HEAT_ARITH_EXACT = 0, /* v = u + r*((ul - 2u) + ur), each operation rounded once
                           to nearest-even, left to right (bit-exact with a plain
                           C evaluation without contraction) */
  HEAT_ARITH_FMA = 1    /* v = fma(r, (ul - 2u) + ur, u): one rounding fewer */
} heat_arith;

/* Create a ring of np partitions x nx points with Eq. 2 coefficient
 * r = (k*dt)/(dx*dx), computed once on the host in binary64.
 *   out   receives the new context (set to NULL on failure).
 *   nx>=1, np>=1, nx*np must not overflow int64; k, dt, dx finite, dx != 0.
 *   r > 1/2 is accepted (explicit Euler is then unstable; not an error).
 * The state is zero until heat_set().  Returns HEAT_EINVAL, HEAT_ENOMEM or
 * HEAT_ECUDA on failure (nothing is leaked). */
int heat_create(heat_ctx **out, int64_t nx, int32_t np, double k, double dt, double dx,
                heat_dtype dtype);

/* Free every device resource of the context (synchronises its stream).  NULL is
 * a no-op. */
void heat_destroy(heat_ctx *c);

/* Load the state from host memory: host_u holds n = np*nx binary64 values in
 * global order (Section 2's initial condition u(0, x_i) is the caller's).  For
 * HEAT_F32C each value is rounded to nearest binary32 on the device.  Resets the
 * step counter to 0.  Synchronous.  n != np*nx -> HEAT_EINVAL. */
int heat_set(heat_ctx *c, const double *host_u, int64_t n);

/* Read the state into host memory (n = np*nx binary64 values; binary32 state is
 * widened exactly).  Synchronises the context's stream first and reports a
 * pending device error, if any, instead of copying. */
int heat_get(heat_ctx *c, double *host_u, int64_t n);

/* Same as heat_set / heat_get with a device pointer (binary64, n elements,
 * 8-byte aligned) instead of a host pointer; the copy is queued on the
 * context's stream (heat_set_device returns without waiting; heat_get_device
 * waits for the stream). */
int heat_set_device(heat_ctx *c, const double *dev_u, int64_t n);
int heat_get_device(heat_ctx *c, double *dev_u, int64_t n);

/* Advance the state by nt >= 0 forward-Euler steps of Eq. 2 (Section 2, with
 * the periodic boundary u(t, x) = u(t, L + x): the neighbours of point 0 and
 * N-1 wrap around the ring) with the current form and arithmetic.  Asynchronous on the context's stream; returns HEAT_EINVAL for
 * nt < 0, HEAT_ESTATE if a device error is pending, HEAT_ECUDA if a launch
 * fails.  Errors found on the device during the run surface at the next
 * synchronising call. */
int heat_run(heat_ctx *c, int64_t nt);

/* Wait for the context's stream and report a pending device error
 * (HEAT_ETIMEOUT) or HEAT_OK.  The pending error is cleared by heat_set(). */
int heat_sync(heat_ctx *c);

/* Queue subsequent work on cuda_stream (a cudaStream_t, e.g. the handle of a
 * torch.cuda.Stream); NULL restores the context's own stream. */
int heat_set_stream(heat_ctx *c, void *cuda_stream);

/* Select the kernel form and, for the blocked forms (HEAT_FORM_PERSIST,
 * HEAT_FORM_TBLOCK, HEAT_FORM_CLUSTER, HEAT_FORM_PERSIST_TB), the temporal
 * block depth T (1..64;
 * 0 = library default: 32 for HEAT_F32C; for HEAT_F64 in the temporal-blocking
 * form 24 on rings below 2^19 points (12 there when integer tiles run at an r
 * that is not a power of two), else 12 when part of the tiles run on the
 * integer pipes, else 8 below 2^22 points and 4 from 2^22 points; in the
 * cluster form 16, or 8 for rings that one cluster holds only at that depth;
 * in the persistent temporal-blocking form 32 for HEAT_F32C, for HEAT_F64 16
 * below 2^19 points, 12 from 2^19 to 2^21 and 16 from 2^21; in the flag-queue
 * form 32 for HEAT_F32C, for HEAT_F64 8 below 2^21 points and 16 from 2^21).
 * The flag-queue form runs at depth 1 when a partition is shorter than T.
 * T is ignored by the plain form.
 * HEAT_FORM_AUTO (the default) is HEAT_FORM_CLUSTER for binary64 rings of at
 * most 6144 points and binary32 rings that one thread-block cluster holds,
 * HEAT_FORM_PERSIST_TB for binary64 rings under the exact reading from 2^18 to
 * 2^26 points, else HEAT_FORM_TBLOCK. */
int heat_set_form(heat_ctx *c, int form, int T);

/* Segmentation of the persistent flag-queue form: 0 = library default
 * (near-equal segments, one per co-resident CTA; at depth 1 interior
 * boundaries fall on 64-point tiles, deeper every segment keeps at least T
 * points);
 * -1 = one segment per partition of nx points, as in the paper's algorithm, when
 * np CTAs can be co-resident (else the default); n > 0 = at most n near-equal
 * segments.  The result does not depend on this choice. */
int heat_set_segments(heat_ctx *c, int segments);

/* Binary64 with HEAT_ARITH_EXACT, temporal-blocking form (either layout):
 * compute `share` of every 32 tiles with integer-pipe binary64 arithmetic
 * instead of the FP64 unit (0..32), or -1 (the default) to let the library
 * choose: with the contiguous layout, for rings of at least 2^18 points, half
 * of the warps take tiles for the integer pipes from the end of the ring while
 * the other half take tiles for the FP64 unit from the start, so the split
 * follows the two engines' speeds; else every tile on the FP64 unit.
 * GB300's FP64 unit runs at 1/64 of the FP32 rate; the integer pipes are idle
 * during the binary64 update, so splitting the tiles between the two raises
 * throughput.  Both paths give the correctly rounded IEEE result, so the state
 * is bitwise the same for every share.  Strided layout: a tile in which a
 * value leaves the integer routines' domain (subnormal or non-finite operands or
 * results, signed zeros) is recomputed on the FP64 unit.  Contiguous layout: a
 * tile runs on the integer pipes only if its values pass a screen (+0, or
 * normal magnitudes within bounds derived from T and r that keep every
 * intermediate result normal), else on the FP64 unit.  For r = +-2^k the
 * contiguous layout's FP64-unit tiles that pass the same screen multiply by
 * moving the exponent with an integer add (three FP64-unit operations per
 * point instead of four; the same bits).  The persistent temporal-blocking
 * form (HEAT_FORM_PERSIST_TB) takes the same setting; there -1 splits each
 * work unit's tiles between the two engines the same way at every ring size.
 * HEAT_EINVAL outside -1..32. */
int heat_set_emulation(heat_ctx *c, int share);

/* The share of 32 tiles the temporal-blocking form computes on the integer
 * pipes for this ring as configured now, into *share: 0..32, or -1 when the
 * library's adaptive split applies.  HEAT_EINVAL for null arguments. */
int heat_get_emulation(const heat_ctx *c, int *share);

/* Binary64 with HEAT_ARITH_EXACT, temporal-blocking form with the strided
 * layout, tiles left on the FP64 unit: move part of each point's update to the
 * integer pipes.  level 0:
 * all four operations (fma for ul - 2u, add, multiply by r, add) on the FP64
 * unit; 1: the multiply by r on the integer pipes (3 FP64 operations per
 * point; for r a power of two the product only moves the exponent); 1 + j
 * (j = 1..16): also the final add, for j/16 of the points (2 FP64 operations
 * there).  Bitwise the same state for every level (every operation is the
 * correctly rounded IEEE result either way). */
int heat_set_split(heat_ctx *c, int level);

/* Register layout of the temporal-blocking form: 0 = strided (lane l holds
 * window points 32k + l; windows staged into shared memory by bulk TMA copies),
 * 1 = contiguous (lane l holds E consecutive points; neighbours inside a lane
 * come from its own registers, so a step needs two shuffles per lane instead of
 * two per point; the default).  The state is bitwise the same for either layout. */
int heat_set_layout(heat_ctx *c, int layout);

/* CUDA graphs for the multi-launch forms (plain, temporal blocking), on by
 * default: the first run with a given (form, T, nt, starting buffer,
 * arithmetic, layout, stream) is captured into a graph, later identical runs
 * replay it.  Runs of more than 8192 launches are not captured. */
int heat_set_graphs(heat_ctx *c, int enable);

/* Select the rounding reading for HEAT_F64 (heat_arith).  HEAT_F32C ignores it. */
int heat_set_arith(heat_ctx *c, int arith);

/* Deterministic FP64 sum of the state into *out (host pointer): a fixed-shape
 * tree, so the value does not depend on timing or on the GPU.  It is the conservation
 * diagnostic: sum(u) is invariant under Eq. 2 on the periodic ring.
 * Synchronous. */
int heat_sum(heat_ctx *c, double *out);

/* Number of steps applied since the last heat_set (the checkpoint counter:
 * heat_get + this count is a checkpoint; heat_set restores). */
int heat_steps(const heat_ctx *c, int64_t *out);

/* What the last heat_run did: the form it used (HEAT_FORM_AUTO resolved), the
 * temporal block depth (1 for the one-step forms), the number of stencil kernel
 * launches it queued, and the persistent forms' segment count.  Any pointer may
 * be NULL. */
int heat_last_run(const heat_ctx *c, int *form, int *T, int64_t *launches, int *segments);

/* Ring geometry and the coefficient actually used. */
int heat_info(const heat_ctx *c, int64_t *nx, int32_t *np, double *r, int *dtype);

/* Device pointer of the current state buffer (dtype elements, global order).
 * Borrowed: valid until the next heat_run/heat_set/heat_destroy. */
int heat_state_ptr(heat_ctx *c, void **dev_ptr);

/* Upper bound, in nanoseconds, on any single device wait for a neighbour's
 * ghost value in the persistent forms (default 2e9).  A wait that runs out
 * stops the run and reports HEAT_ETIMEOUT. */
int heat_set_wait_limit(heat_ctx *c, int64_t ns);

/* Test hook (host-side fault injection): in the next persistent run, the CTA
 * owning segment `segment` stops publishing its edge values from step
 * `from_step` on, so its neighbours' bounded waits run out and the run ends with
 * HEAT_ETIMEOUT while every kernel still returns normally.  segment < 0
 * disables the hook.  No GPU fault or trap is involved. */
int heat_inject_stall(heat_ctx *c, int32_t segment, int64_t from_step);

/* ---------------------------------------------------------------------------
 * Batched rings: many independent instances of Section 2's problem, each with
 * its own size, partition count, coefficient and step count, held in one
 * device arena and advanced together by one persistent launch.  A ring's
 * result is bitwise the one heat_run gives for it alone (binary64) or the one
 * the temporal-blocking form gives with the same block depth (HEAT_F32C).
 *
 * The batch's kernel runs over a work table of units (level b, ring, tile): a
 * ring of n points is cut into near-equal warp tiles (of at most the warp
 * window minus 2T points); level b advances a tile by T steps (fewer at the
 * ring's last level); warps claim units in level order, and a unit waits
 * (bounded) until its tile and the two neighbouring tiles have finished level
 * b-1.  T and the warp window come from heat_batch_set_tuning or
 * heat_batch_autotune.
 * ------------------------------------------------------------------------- */
typedef struct heat_batch heat_batch; /* opaque, library-owned */

/* Arena for `capacity_points` ring points (two buffers of that many elements of
 * dtype, allocated now).  Each ring takes its n points rounded up to 64. */
int heat_batch_create(heat_batch **out, int64_t capacity_points, heat_dtype dtype);

/* Free the arena and tables (synchronises).  NULL is a no-op. */
void heat_batch_destroy(heat_batch *b);

/* Admit a ring of np x nx points with coefficient r = k*dt/dx^2 that will
 * advance nt steps, initial state host_u (n = nx*np binary64 values, global
 * order).  *ring_id receives its handle.  HEAT_ENOMEM when the arena has no
 * contiguous room (the caller may wait for rings to be removed: admission by
 * free device memory).  Synchronous copy. */
int heat_batch_add(heat_batch *b, int64_t nx, int32_t np, double k, double dt, double dx, int64_t nt,
                   const double *host_u, int32_t *ring_id);

/* Same with the initial state in device memory (n binary64 values, 8-byte
 * aligned); the copy is queued on the batch's stream (no wait). */
int heat_batch_add_device(heat_batch *b, int64_t nx, int32_t np, double k, double dt, double dx, int64_t nt,
                          const double *dev_u, int32_t *ring_id);

/* Advance every ring that has steps left by min(steps left, max_steps) steps
 * (max_steps <= 0: all remaining steps) in one persistent launch.
 * Asynchronous on the batch's stream; device errors surface at heat_batch_sync
 * or heat_batch_get. */
int heat_batch_run(heat_batch *b, int64_t max_steps);

/* Wait for the batch's stream; HEAT_ETIMEOUT if a dependency wait ran out. */
int heat_batch_sync(heat_batch *b);

/* Steps done and steps left of a ring. */
int heat_batch_query(const heat_batch *b, int32_t ring_id, int64_t *steps_done, int64_t *steps_left);

/* Copy a ring's current state to host memory (n binary64 values; synchronises). */
int heat_batch_get(heat_batch *b, int32_t ring_id, double *host_u, int64_t n);

/* Queue a copy of a ring's current state into device memory (n binary64
 * values) on the batch's stream; no wait, no status check beyond a pending
 * error seen at an earlier sync. */
int heat_batch_get_device(heat_batch *b, int32_t ring_id, double *dev_u, int64_t n);

/* Release a ring's arena space (its id becomes invalid).  Does not wait: work
 * queued on the batch's stream before the call (a run, a heat_batch_get_device
 * copy of the ring) still reads the old space, and every later use of that space
 * is queued behind it on the same stream. */
int heat_batch_remove(heat_batch *b, int32_t ring_id);

/* Temporal block depth T (1..64) and warp window in points: the kernel has
 * three windows, 128, 256 and 512 binary64 points (256, 512 and 1024 binary32
 * points); a request takes the widest of them not above it, at least the
 * narrowest.  0 keeps the current value (defaults: T = 8 for binary64, 32 for
 * HEAT_F32C; the widest window).  A run widens the window while a tile would
 * keep fewer than 2T output points. */
int heat_batch_set_tuning(heat_batch *b, int T, int64_t window_points);

/* Pick T and the warp window by timing one level of the current rings for each
 * candidate (the rings' states are not changed: one level only writes the idle
 * buffer).  The choice is cached in the file named by the environment variable
 * HEAT_TUNE_CACHE, if set, keyed by dtype and a coarse description of the
 * batch.  Synchronous. */
int heat_batch_autotune(heat_batch *b, int *T_out, int64_t *window_points_out);

/* Queue subsequent work on cuda_stream (NULL: the batch's own stream). */
int heat_batch_set_stream(heat_batch *b, void *cuda_stream);

/* CUDA graphs for batch runs, on by default: a run's stream operations (table
 * upload, counter resets, launch) are captured once and replayed while their
 * shape is unchanged, e.g. for a fixed batch run again after heat_batch_restore. */
int heat_batch_set_graphs(heat_batch *b, int enable);

/* Binary64 batches (exact reading): `share` of every 32 tiles of each work unit
 * computed on the integer pipes instead of the FP64 unit (0..32), or -1 (the
 * default) for the library's choice: within each unit, half of the warps take
 * tiles for the integer pipes from the end and the others tiles for the FP64
 * unit from the start, so the split follows the two engines' speeds.  A tile
 * runs on the integer pipes only if its values pass the screen described at
 * heat_set_emulation; the state is bitwise the same for every share.
 * HEAT_EINVAL outside -1..32. */
int heat_batch_set_emulation(heat_batch *b, int share);

/* Upper bound, in nanoseconds, on a unit's wait for its neighbours' previous
 * level (default 5e9).  A wait that runs out stops the launch and reports
 * HEAT_ETIMEOUT at the next heat_batch_sync / heat_batch_get. */
int heat_batch_set_wait_limit(heat_batch *b, int64_t ns);

/* Test hook (host-side fault injection): in later runs, tile `segment` of
 * ring `ring_id` stops publishing its completion from level `from_level` on,
 * so the units that depend on it run out of their bounded waits and the run
 * ends with HEAT_ETIMEOUT; every kernel returns normally.  A ring id that is
 * not live (e.g. -1) disables the hook. */
int heat_batch_inject_stall(heat_batch *b, int32_t ring_id, int64_t segment, int64_t from_level);

/* Cap the batch kernel's CTAs per SM (0: as many as fit).  The launch needs no
 * co-residency, so two batches on two streams with caps that together fit an
 * SM run side by side: a binary64 batch (FP64 unit) and a binary32 batch
 * (FP32 and integer pipes) then share every SM. */
int heat_batch_set_ctas_per_sm(heat_batch *b, int ctas_per_sm);

/* Checkpoint of every live ring (its state and step count) into a device copy
 * the batch keeps; heat_batch_restore puts those states back (and clears a
 * pending device error).  Rings added after the save are left as they are. */
int heat_batch_save(heat_batch *b);
int heat_batch_restore(heat_batch *b);

/* Live rings, free points in the arena (largest contiguous block), and the
 * point-steps the last heat_batch_run queued. */
int heat_batch_info(const heat_batch *b, int32_t *live_rings, int64_t *largest_free_points,
                    int64_t *last_point_steps);

/* ---------------------------------------------------------------------------
 * Request server: continuous batching inside one running kernel.  Requests
 * (independent instances of Section 2's problem, each its own size, coefficient
 * and step count) are admitted into a device arena and a slot table while a
 * persistent kernel runs; its warps find admitted requests in the slot table,
 * claim their (level, warp tile) units in level order from each request's own
 * counter, wait (bounded) on the neighbouring tiles' completion counters as in
 * the batched-ring kernel, and mark a request complete in host-mapped memory
 * when its last unit is done.  A request submitted while others run joins the
 * running kernel at once: no launch boundary, no host tick.  A request's result
 * is bitwise the one heat_run gives for it alone (binary64) or the one the
 * temporal-blocking form gives with the server's block depth (HEAT_F32C).
 * The server kernel ends by itself, all of its warps together, once a warp
 * has found no admitted request with units left for `idle_ns`;
 * heat_server_submit (or heat_server_poll, while requests are in flight)
 * starts it again.  The running kernel fills most of each SM, so work the
 * caller launches beside it waits for room: the initial states passed to
 * heat_server_submit should be ready before the call, not computed by a
 * kernel per request.  While it runs, a device-wide synchronisation
 * (cudaDeviceSynchronize) waits for it to end: synchronise streams instead.  The paper has no serving layer; this is the library's (it
 * serves the paper's problem).
 * ------------------------------------------------------------------------- */
typedef struct heat_server heat_server; /* opaque, library-owned */

/* Server for requests of dtype with room for `capacity_points` ring points
 * (two arena buffers, allocated now) and at most `max_requests` (1..65536)
 * requests in flight; T (1..64, 0: 16 for binary64, 32 for HEAT_F32C) is its
 * temporal block depth (warp windows of 512 points).  ctas_per_sm caps the
 * server kernel's CTAs per SM (0: one fewer than fit; the cap is always below
 * what fits, so that the small copy and publish kernels of admission run beside
 * it), so that two servers (binary64 and binary32) can share every SM. */
int heat_server_create(heat_server **out, int64_t capacity_points, heat_dtype dtype, int32_t max_requests, int T,
                       int ctas_per_sm);

/* Stop the server kernel (it finishes its current units), wait for it and free
 * everything.  NULL is a no-op. */
void heat_server_destroy(heat_server *s);

/* Admit a ring of n points with coefficient r = k*dt/dx^2 that advances nt >= 1
 * steps from the initial state dev_u (n binary64 values in device memory,
 * 8-byte aligned).  The copy into the arena is queued on the server's copy
 * stream, which does not wait for other streams: dev_u must hold its values
 * when the call is made and stay unchanged until the request is reported
 * complete.  The request is published to the running kernel behind the copy
 * (and the kernel launched if it is not running).  *req_id receives the
 * request's handle.  HEAT_ENOMEM when the arena or the slot table has no room
 * (the caller may retry after releasing completed requests); HEAT_ESTATE after
 * a device error. */
int heat_server_submit(heat_server *s, int64_t n, double k, double dt, double dx, int64_t nt, const double *dev_u,
                       int32_t *req_id);

/* Requests completed since the last call, without waiting: up to `max` ids into
 * done_ids, their number into *count.  HEAT_ETIMEOUT if a bounded wait of the
 * server kernel ran out (the server then refuses submissions). */
int heat_server_poll(heat_server *s, int32_t *done_ids, int32_t max, int32_t *count);

/* Queue a copy of a completed request's final state (n binary64 values) into
 * device memory on the server's copy stream; `cuda_event`, if not NULL, is a
 * cudaEvent_t recorded behind the copy.  HEAT_ESTATE if the request is not
 * complete. */
int heat_server_get_device(heat_server *s, int32_t req_id, double *dev_u, int64_t n, void *cuda_event);

/* Free a completed request's slot and arena space (after copies queued on the
 * copy stream). */
int heat_server_release(heat_server *s, int32_t req_id);

/* Point-steps of the requests completed so far, requests in flight, whether
 * the server kernel is running, and how many times it has been launched.  Any
 * pointer may be NULL. */
int heat_server_info(const heat_server *s, int64_t *point_steps, int32_t *in_flight, int *running,
                     int64_t *launches);

/* Upper bound, in nanoseconds, on a unit's wait for its neighbours (default
 * 5e9) and on the kernel's idle time before it ends (default 2e8). */
int heat_server_set_limits(heat_server *s, int64_t wait_ns, int64_t idle_ns);

/* Allocation-free stepper for callers that cannot allocate device memory
 * (inside CUDA graph capture, in real-time loops that must stay off the
 * allocator, or under another framework's memory pool).  The paper has no
 * counterpart: this is a packaging of the plain form.
 *   dev_u0  device input, n binary64 values in ring order, only read;
 *   dev_u   device output, n binary64 values, receives u^nt;
 *           both 16-byte aligned and not overlapping;
 *   n       1 .. 1048576 points (larger rings -> HEAT_EINVAL: the library's one
 *           fixed scratch array holds 2^20 values);
 *   k, dt, dx, arith   as for heat_create / heat_set_arith;
 *   cuda_stream        cudaStream_t the steps are queued on (NULL = default);
 *                      it must belong to the current device (a stream of
 *                      another device -> HEAT_EINVAL).
 * Queues nt launches and returns without waiting.  It calls no cudaMalloc,
 * cudaFree or other allocating routine: the buffer a multi-step run needs
 * besides input and output is a fixed 8 MiB device array that every GPU loading
 * this library holds until the process exits.  The first call on each device
 * looks up that array's device address (cudaGetSymbolAddress) with the device
 * current and loads the kernels of both arithmetic readings; make that first
 * call, in either reading, before any stream capture.  All calls on a device
 * share the array, so calls whose work overlaps on the GPU (two streams, two
 * host threads) race and must be ordered by the caller.
 * HEAT_ECUDA: a CUDA error was already pending on the calling thread (reported,
 * not cleared; nothing queued), or a launch failed part-way, in which case the
 * steps queued before it still run and dev_u is undefined. */
int heat_run_noalloc(const double *dev_u0, double *dev_u, int64_t n, double k, double dt, double dx,
                     int64_t nt, int arith, void *cuda_stream);

/* Measured issue rates of the engines the binary64 update runs on, for roofline
 * denominators (the paper has no counterpart: it measures CPUs).  Three probe
 * kernels run on the current device, on cuda_stream (NULL = default stream),
 * each on a full-occupancy grid of independent dependency chains, timed with
 * CUDA events after one untimed launch: binary64 fused multiply-adds, binary64
 * adds, and 32-bit bitwise majorities (LOP3, ALU-pipe instructions).  Results are
 * lane operations per second; any pointer may be NULL.  Synchronous; allocates
 * and frees a small device buffer.  HEAT_ECUDA if a launch fails. */
int heat_probe_pipes(void *cuda_stream, double *dfma_lane_ops_per_s, double *dadd_lane_ops_per_s,
                     double *alu_lane_ops_per_s);

/* Static text for a status code. */
const char *heat_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* HEAT_H */
