/*
 * links.h -- C ABI of the GB300 batched planar-linkage simulator.
 *
 * Method: LINKS (Nobari, Srivastava, Gutfreund, Ahmed; arXiv 2208.14567).
 * A mechanism is an undirected graph over n joints given by an n x n 0/1
 * adjacency matrix, a type per joint (0 fixed, 1 simple, 2 actuated) and the
 * initial joint positions (Sec. "Mechanism Representation").  It is simulated
 * over T equally spaced positions of one full actuator turn (Sec. "Dataset
 * Features & Statistics", item Simulation Data) with the graphical solver: from the known
 * joints (fixed + actuated), repeatedly solve a joint with two known neighbours
 * by intersecting two circles (Sec. "Graphical Simulator", Fig. "solver").  A
 * candidate is valid when the actuator completes the turn without locking
 * (Sec. "Finding Valid Initial Positions", Infeasibility rule).
 *
 * Conventions for every call:
 *   - the return value is a LINKS_* status; 0 is success; no exception or
 *     abort crosses this boundary; links_last_error() describes the last
 *     failure of the calling thread;
 *   - "device" pointers are CUDA device memory owned by the caller (any
 *     allocator); "host" pointers are caller-owned host memory;
 *   - calls taking device pointers are asynchronous on the context's stream
 *     and make no allocation (except the context workspace, which the path
 *     calls grow on demand and links_workspace_reserve sizes ahead), so a
 *     sequence of them can be captured in a CUDA graph between
 *     links_capture_begin and links_capture_end;
 *   - the library owns contexts, plans, graphs and compiled topology screens
 *     and frees them in the matching *_free / links_destroy call.
 */
#ifndef LINKS_H
#define LINKS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LINKS_API __attribute__((visibility("default")))
#else
#define LINKS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Call statuses. */
#define LINKS_OK 0
#define LINKS_EINVAL 1     /* bad argument: null pointer, size out of range, unknown enum */
#define LINKS_ECUDA 2      /* a CUDA runtime call failed (text in links_last_error) */
#define LINKS_ENOMEM 3     /* allocation failed */
#define LINKS_ECAPACITY 4  /* a batch larger than the plan's capacity */
#define LINKS_EBUSY 5      /* serving ring full; retry later */
#define LINKS_ETIMEDOUT 6  /* a bounded wait ran out */
#define LINKS_ESTATE 7     /* call not valid in the current state */
#define LINKS_EDEVICE 8    /* a kernel raised its error word (see links_sync) */

/* Per-mechanism plan statuses written by links_plan_build*.  A mechanism that
 * is not OK is not simulated: valid = 0, lock_step = -2. */
#define LINKS_MECH_OK 0
#define LINKS_MECH_BAD_SIZE 1          /* n < 2 or n > n_max */
#define LINKS_MECH_BAD_TYPE 2          /* a type outside {0,1,2} */
#define LINKS_MECH_BAD_ADJ 3           /* adjacency not symmetric or a self-loop */
#define LINKS_MECH_NO_MOTOR 4          /* not exactly one actuated joint */
#define LINKS_MECH_NO_PIVOT 5          /* actuated joint has no fixed neighbour */
#define LINKS_MECH_NOT_DYAD_SOLVABLE 6 /* complex loop or dangling joint: the solver stalls */
#define LINKS_MECH_OVERCONSTRAINED 7   /* > 2 known neighbours, or links beyond 2 per simple joint */

/* Position dtype, precision and output mode selectors. */
#define LINKS_F32 0
#define LINKS_F64 1
#define LINKS_PLAIN_F64 0 /* one thread per mechanism, native FP64 throughout */
#define LINKS_MIXED 1     /* FP32 screen with certified lock decisions; double-word
                             FP32 where FP32 cannot certify; double-word trajectories */
#define LINKS_OUT_FULL 0       /* rows = all B mechanisms */
#define LINKS_OUT_VALID_ONLY 1 /* rows = valid mechanisms in index order, compacted */

#define LINKS_MAX_JOINTS 32
#define LINKS_MAX_T 32767

typedef struct links_ctx_s* links_ctx;
typedef struct links_plan_s* links_plan;
typedef struct links_graph_s* links_graph;
typedef struct links_topo_s* links_topo;

/* Text of the calling thread's last failure ("" if none).  Static storage. */
LINKS_API const char* links_last_error(void);
/* Name of a LINKS_* call status. */
LINKS_API const char* links_strerror(int status);

/* Context on CUDA device `device` issuing work on `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream).  The library owns *out. */
LINKS_API int links_create(links_ctx* out, int device, void* cuda_stream);
LINKS_API int links_destroy(links_ctx ctx);
/* Later calls on ctx issue work on this stream. */
LINKS_API int links_set_stream(links_ctx ctx, void* cuda_stream);
/* Waits for the stream, then reads and clears the device error word:
 * LINKS_EDEVICE if a kernel raised it since the last links_sync. */
LINKS_API int links_sync(links_ctx ctx);
/* Allocates the per-T actuator tables (cos/sin of 2*pi*t/T in FP64 and as
 * float pairs).  Called implicitly by links_simulate; call it before a graph
 * capture that uses a T not simulated before. */
LINKS_API int links_prepare(links_ctx ctx, int T);

/* Plan storage for up to `capacity` mechanisms of at most n_max joints
 * (2 <= n_max <= LINKS_MAX_JOINTS).  Allocates device memory; the library owns
 * the plan. */
LINKS_API int links_plan_create(links_ctx ctx, int64_t capacity, int n_max, links_plan* out);
LINKS_API int links_plan_free(links_plan plan);

/* Solve order of B mechanisms (Sec. "Graphical Simulator"; the found path is
 * reused for every actuator position, Sec. "Graphical Simulator", last
 * paragraph).  Device inputs, row-major, padded to the plan's n_max:
 *   n_joints [B] int32, adj [B,n_max,n_max] uint8 (nonzero = link),
 *   type [B,n_max] int8 (0 fixed, 1 simple, 2 actuated), pos0 [B,n_max,2]
 *   float32 or float64 (pos_dtype).
 * status_out [B] int32 (device, may be NULL) receives LINKS_MECH_*.
 * Rules: the crank pivot is the lowest-index fixed neighbour of the actuated
 * joint; the lowest-index unknown joint with >= 2 known neighbours is solved
 * next, with the branch (orientation sign) of the initial positions.
 * Asynchronous; inputs may be reused once the stream has passed this call. */
LINKS_API int links_plan_build(links_ctx ctx, links_plan plan, int64_t B, const int32_t* n_joints,
                     const uint8_t* adj, const int8_t* type, const void* pos0, int pos_dtype,
                     int32_t* status_out);

/* links_plan_build with the adjacency given as neighbour bit masks (the same matrix,
 * one bit per entry): nbr [B, n_max] uint32 (device), bit c of nbr[b][a] set when
 * joints a and c are linked; bits at c >= n_joints[b] are ignored.  The other inputs,
 * the rules and the plan are those of links_plan_build (the same plan to the bit); the
 * masks are a fifth of the bytes of the uint8 matrix at n_max 20 and need no
 * conversion on the device.  Asynchronous.  LINKS_EINVAL / LINKS_ECAPACITY as
 * links_plan_build. */
LINKS_API int links_plan_build_masks(links_ctx ctx, links_plan plan, int64_t B, const int32_t* n_joints,
                                     const uint32_t* nbr, const int8_t* type, const void* pos0, int pos_dtype,
                                     int32_t* status_out);

/* Same rules, same result, computed by host threads from HOST inputs; the plan
 * is uploaded on the context's stream.  status_out [B] is host memory.
 * Synchronous (returns after the upload completed). */
LINKS_API int links_plan_build_host(links_ctx ctx, links_plan plan, int64_t B, const int32_t* n_joints,
                          const uint8_t* adj, const int8_t* type, const void* pos0, int pos_dtype,
                          int32_t* status_out);

/* Mechanisms in the last build, the plan's n_max and its capacity. */
LINKS_API int links_plan_info(links_plan plan, int64_t* B, int* n_max, int64_t* capacity);


/* Copies the plans of mechanisms [b0, b0 + count) to HOST memory, for inspection:
 *   topo [count, 6 + 3 (n_max - 2)] int32: status, n, motor joint, pivot joint,
 *       coupler joint, dyad count nd, then per dyad (k, i, j) as joint indices with
 *       (i, j) in the order that makes the solved branch the "+" one, i.e.
 *       (p_j - p_i) x (p_k - p_i) >= 0 in the initial configuration;
 *   lengths [count, 2 (n_max - 2)] float64 (may be NULL): r1^2 = |p_k - p_i|^2 and
 *       r2^2 = |p_k - p_j|^2 per dyad (double-word values widened to FP64).
 * Synchronous. */
LINKS_API int links_plan_export(links_plan plan, int64_t b0, int64_t count, int32_t* topo,
                                double* lengths);

/* Simulate the planned mechanisms over T actuator steps, crank angle 2*pi*t/T
 * counter-clockwise from the initial crank (t = 0..T-1).
 * Device outputs (all caller-owned; any of traj, path may be NULL):
 *   valid [B] uint8: 1 = no lock over the T steps;
 *   lock_step [B] int16: first locking step, -1 none, -2 not simulated;
 *   min_disc [B] float32: min over the dyads of the steps before the lock of
 *       q = D / (4 r1^2 r2^2) = sin^2 of the angle at the solved joint, where
 *       D = 4 d^2 r1^2 - (d^2 + r1^2 - r2^2)^2 (NaN if not simulated);
 *   traj [rows,n_max,T,2] and path [rows,T,2] (coupler = last joint of the
 *       solve order): float64 for LINKS_PLAIN_F64, float32 for LINKS_MIXED;
 *       NaN from the locking step on and for joints >= n.
 * out_mode LINKS_OUT_FULL: rows = B.  LINKS_OUT_VALID_ONLY: rows = valid
 *   mechanisms in increasing index; out_index [out_capacity] int32 gets each
 *   row's mechanism index, *n_out (device int32) the number of valid ones;
 *   rows beyond out_capacity are not written.
 * A step locks when a dyad has D <= 0 (no intersection) -- locking is a result,
 * not an error.  Asynchronous. */
LINKS_API int links_simulate(links_ctx ctx, links_plan plan, int T, int precision, int out_mode,
                   void* traj, void* path, uint8_t* valid, int16_t* lock_step, float* min_disc,
                   int32_t* out_index, int64_t out_capacity, int32_t* n_out);

/* links_simulate in LINKS_OUT_VALID_ONLY mode with the rows' trajectories packed by
 * joint count (no counterpart in the paper: the valid rows without their padding
 * joints).  Row r (mechanism out_index[r], n_r joints) holds joint j < n_r at
 * traj[(row_offset[r] + j) * T + t] (float32 pairs for LINKS_MIXED, float64 pairs for
 * LINKS_PLAIN_F64; the values those of links_simulate's row r, joint j).
 * row_offset [out_capacity + 1] int64 (device) receives the exclusive prefix of n_r
 * over the rows and, at index rows = min(*n_out, out_capacity), their total.  traj
 * (device, may be NULL) holds traj_capacity joint rows of T points; a row that does not
 * fit entirely is not written (its path is).  path [out_capacity, T, 2], out_index,
 * *n_out, valid, lock_step and min_disc as in links_simulate.  Nothing is written for
 * joints >= n_r.  Asynchronous (graph-capturable).  LINKS_EINVAL for bad arguments
 * (row_offset is required). */
LINKS_API int links_simulate_packed(links_ctx ctx, links_plan plan, int T, int precision, void* traj,
                                    int64_t traj_capacity, void* path, uint8_t* valid, int16_t* lock_step,
                                    float* min_disc, int32_t* out_index, int64_t* row_offset,
                                    int64_t out_capacity, int32_t* n_out);

/* Two-stage screen (Sec. "Finding Valid Initial Positions", paragraph on low fidelity
 * evaluations): LINKS_MIXED simulation of every OK mechanism on the coarse grid of
 * T_low actuator positions, then on the full grid of T positions only for the
 * mechanisms valid on the coarse one, then the valid rows as in links_simulate with
 * LINKS_OUT_VALID_ONLY (traj [out_capacity, n_max, T, 2], path [out_capacity, T, 2],
 * out_index, *n_out; all device).  T_low must divide T, so the coarse angles
 * 2 pi t / T_low are fine-grid angles: a coarse lock is a fine lock, and valid[] is
 * exactly the full-grid verdict.  For the mechanisms the coarse pass rejects,
 * lock_step is that locking step scaled to the fine grid (a locking step, not
 * necessarily the first) and min_disc covers the coarse steps before it; for the
 * others all outputs are those of links_simulate.  *n_low_valid (device int32, may be
 * NULL) receives the number valid on the coarse grid, so n_low_valid - *n_out counts
 * the coarse grid's false valids.  Asynchronous.  LINKS_EINVAL for bad arguments. */
LINKS_API int links_simulate_two_stage(links_ctx ctx, links_plan plan, int T, int T_low, float* traj, float* path,
                                       uint8_t* valid, int16_t* lock_step, float* min_disc, int32_t* out_index,
                                       int64_t out_capacity, int32_t* n_out, int32_t* n_low_valid);

/* Census of the LINKS_MIXED emit (the work its precision design does; no
 * counterpart in the paper): runs the emit's FP32 chain and forward error bound
 * (Sec. "Graphical Simulator" steps) over the rows links_simulate wrote for this plan
 * at T -- every OK mechanism's steps before its lock (LINKS_OUT_FULL, from lock_step
 * [B] device) or the first min(n_out, out_capacity) rows of out_index (device;
 * LINKS_OUT_VALID_ONLY, all T steps) -- writing nothing, and copies to out[3] (host):
 * [0] steps computed, [1] steps whose bound exceeds the tolerance, which the emit
 * recomputes in double-word, [2] the same in dyad-steps.  The decisions are the
 * emit's own (same arithmetic on the same inputs).  Synchronises the context's stream.
 * LINKS_EINVAL for bad arguments. */
LINKS_API int links_emit_census(links_ctx ctx, links_plan plan, int T, int out_mode, const int16_t* lock_step,
                                const int32_t* out_index, int64_t out_capacity, int64_t* out);

/* Path normalisation (Sec. "Dataset Curation & Processing"; the configured variant):
 * for each of M curves of T points (device float32 [M,T,2] in, [M,T,2] out, may
 * alias): subtract the centroid, scale to unit RMS radius, rotate the major axis of
 * the 2x2 covariance onto +x, choosing of the two such rotations the one with
 * sum(x^3) >= 0; an isotropic covariance is not rotated; equal points give zeros.
 * 1 <= T <= 1024.  Asynchronous. */
LINKS_API int links_normalize(links_ctx ctx, int64_t M, int T, const float* curves, float* out);

/* The paper's own path normalisation (Sec. "Dataset Curation & Processing"): the two
 * points of a curve farthest apart, (a, b) with a < b (the first such pair in (a, b)
 * order on ties, in float32), become a horizontal line of length 1 from a to b, and the
 * curve's bounding box is centred at (0.5, 0.5); a curve of equal points becomes
 * (0.5, 0.5).  M curves of T points (device float32 [M,T,2] in, [M,T,2] out, not
 * aliased; 1 <= T <= 256).  pair [M,2] int32 (device, may be NULL) receives (a, b);
 * circ_var [M] float32 (device, may be NULL) the variance of the normalised points'
 * distances from (0.5, 0.5), which the paper's curation compares with 5e-4 to find
 * circles.  Asynchronous.  LINKS_EINVAL for bad arguments. */
LINKS_API int links_normalize_maxline(links_ctx ctx, int64_t M, int T, const float* curves, float* out,
                                      int32_t* pair, float* circ_var);

/* Bidirectional chamfer retrieval (Sec. "A Case Study of Mechanism Retrieval"):
 * CD(P, C) = mean over p in P of min_c |p - c| + mean over c in C of min_p |c - p|
 * (Euclidean), for Q query curves against M database curves of T points each
 * (device float32 [Q,T,2] and [M,T,2]; 1 <= T <= 256).  Writes the k smallest per
 * query (1 <= k <= 32), ascending, ties to the lower database index: idx [Q,k]
 * int32 (-1 past M) and dist [Q,k] float32 (device).  Uses the context's workspace
 * (Q x chunks x k x 8 bytes, plus Q x 7220 bytes of distance tables with pruning on,
 * chunks <= 8 x SMs / ceil(Q/8) + 1; grown on demand, so reserve it with
 * links_workspace_reserve before a graph capture).  Asynchronous. */
LINKS_API int links_chamfer_topk(links_ctx ctx, int Q, int64_t M, int T, const float* queries,
                                 const float* db, int k, int32_t* idx, float* dist);
/* The paper's retrieval (Sec. "A Case Study of Mechanism Retrieval": the curated
 * database is shuffled and read until three curves lie within the chamfer cut-off of
 * the target).  For each of the Q queries, going through the database in the scan
 * order `order` (device, L int32 entries: position r reads database curve order[r];
 * normally a permutation of 0..M-1), the first k curves whose chamfer distance (as
 * in links_chamfer_topk) is below `threshold`.  Outputs (device, caller-owned):
 * idx [Q,k] int32 database curves in scan order, -1 past the hits found; dist [Q,k]
 * float32 their distances, +inf past the hits.  A distance within FP32 rounding of
 * the threshold is recomputed in FP64 and the decision taken on that value.  The
 * chunks of the scan run in parallel; a chunk stops reading once every query has k
 * hits at earlier positions, which changes only the work.  Uses the workspace as
 * links_chamfer_topk (with up to four times as many chunks) plus Q x 4 bytes.
 * Asynchronous.  LINKS_EINVAL for a NULL pointer, Q, M, T, k out of range
 * (as links_chamfer_topk), L outside [0, 2^31 - 1) or a NaN threshold; an order
 * entry outside [0, M) is skipped and raises bit 2 of the device error word
 * (LINKS_EDEVICE from links_sync). */
LINKS_API int links_chamfer_first_under(links_ctx ctx, int Q, int64_t M, int T, const float* queries,
                                        const float* db, int64_t L, const int32_t* order, double threshold,
                                        int k, int32_t* idx, float* dist);
/* ---- Topology-specialised screen (Sec. "Computational Cost of Simulations": the paper
 * vectorises its solver per topology; Sec. "Graphical Simulator": the solve path is
 * found once and serves every position sample).  links_topo_create plans the topology given by one mechanism's n joints,
 * adj [n_max, n_max] and type [n_max] (HOST memory, the layout of links_plan_build),
 * writes CUDA source for its solve path (joint positions and error bounds in
 * registers, parent slots as compile-time names), compiles it for sm_103a with NVRTC
 * and loads it on the context's device; synchronous (tens to hundreds of ms).
 * lanes: steps of one mechanism computed side by side (a group of 8, 16 or 32 lanes;
 * 0 chooses by the number of dyads: up to 3 -> 8, up to 6 -> 16, more -> 32). 
 * LINKS_EINVAL for bad sizes or lanes, or a topology that does not plan (status in the text),
 * LINKS_ECUDA if the compilation or the load fails. */
LINKS_API int links_topo_create(links_ctx ctx, int n, int n_max, const uint8_t* adj, const int8_t* type,
                                int lanes, links_topo* out);
/* The CUDA source links_topo_create compiles for that topology with lanes = 0 (host, no device
 * needed; it includes the library's step.cuh, which the library embeds):
 * NUL-terminated into buf (cap bytes, truncated if shorter), *len (may be NULL) the
 * size it needs including the NUL.  LINKS_EINVAL as links_topo_create. */
LINKS_API int links_topo_source(int n, int n_max, const uint8_t* adj, const int8_t* type, char* buf, size_t cap,
                                size_t* len);
/* Fixed joints and dyads of the compiled solve path, and the time create took. */
LINKS_API int links_topo_info(links_topo topo, int* n_fixed, int* n_dyads, double* compile_ms);
LINKS_API int links_topo_free(links_topo topo);
/* links_simulate with precision LINKS_MIXED (same arguments and outputs), its screen
 * first run by the topology's kernel: every mechanism whose plan follows the compiled
 * path gets its flags, lock step and min_disc from it (the generic screen's values:
 * the same operations in the same order, uncertain steps decided by the same
 * double-word chain); the others go to the generic screen, *n_escaped (device
 * int32, may be NULL) their count.
 * Compaction and emit follow as in links_simulate.  Asynchronous.  LINKS_EINVAL as
 * links_simulate, or for a topology with more joints than the plan's n_max. */
LINKS_API int links_simulate_topology(links_ctx ctx, links_plan plan, links_topo topo, int T, int out_mode,
                                      float* traj, float* path, uint8_t* valid, int16_t* lock_step,
                                      float* min_disc, int32_t* out_index, int64_t out_capacity,
                                      int32_t* n_out, int32_t* n_escaped);

/* The paper's dataset curation (Sec. "Dataset Curation & Processing").  For every
 * joint j of every row r of traj [R, n_max, T, 2] float32 (device; the layout of
 * links_simulate's trajectories, row r belonging to mechanism row_index[r], or to
 * mechanism r when row_index is NULL), given the mechanisms' n_joints [B] int32,
 * adj [B, n_max, n_max] uint8 and type [B, n_max] int8 (device; the layout of
 * links_plan_build):
 *   a joint below n_joints that is not fixed has a path; its path is normalised as
 *   links_normalize_maxline does; it is an arc if the joint is linked to a fixed
 *   joint and a circle if its circle statistic is below circle_var (the paper uses
 *   5e-4); a path that is neither is kept, and an arc or a circle is kept when
 *   draw(b * n_max + j) < keep_rate (the paper keeps 0.5%), where draw(i) is output
 *   i (from 0) of splitmix64 started at `seed`, as (z >> 11) * 2^-53.
 * Outputs (device, caller-owned): flags [R, n_max] uint8 (bit 0 path, bit 1 arc,
 * bit 2 circle, bit 3 kept); circ_var [R, n_max] float32 and pair [R, n_max, 2]
 * int32 (the normalising pair) may be NULL; kept_index [kept_capacity] int32 the
 * entries r * n_max + j of the kept paths in increasing order, *n_kept (device)
 * their count (entries past kept_capacity are dropped); kept_paths
 * [kept_capacity, T, 2] float32 (may be NULL) their normalised paths.  Uses the
 * workspace (R x n_max x 8 bytes when pair is NULL, plus R x n_max / 256 bytes).
 * Asynchronous.  LINKS_EINVAL for a NULL pointer, R, B or kept_capacity negative,
 * n_max outside [1, 64], T outside [1, 256], R x n_max >= 2^31 or a NaN
 * threshold; a row index outside [0, B) gives that row no paths and raises bit 2
 * of the device error word (LINKS_EDEVICE from links_sync). */
LINKS_API int links_curate_paths(links_ctx ctx, int64_t R, int n_max, int T, const float* traj,
                                 const int32_t* row_index, int64_t B, const int32_t* n_joints,
                                 const uint8_t* adj, const int8_t* type, double circle_var, double keep_rate,
                                 uint64_t seed, uint8_t* flags, float* circ_var, int32_t* pair,
                                 int32_t* kept_index, float* kept_paths, int64_t kept_capacity,
                                 int32_t* n_kept);
/* Switches the exact pruning of links_chamfer_topk and links_chamfer_first_under on
 * (1, default) or off (0).  With it on, the column term of each database curve's CD
 * is first bounded from below through a table of the query's distance field
 * (DT(c) >= DT(v) - |c - v| for a grid node v), and the exact computation stops once
 * its partial column sum passes the pruning distance: the smallest k-th distance
 * found so far for the query (in any database chunk) for the top-k, the threshold
 * for the first-k scan.  Curves ruled out either way cannot enter the result, so it
 * is the same bit for bit, only the work differs.  LINKS_EINVAL for a NULL ctx or a
 * flag other than 0 or 1. */
LINKS_API int links_set_chamfer_prune(links_ctx ctx, int on);
/* Makes the context's workspace at least `bytes` large (allocates; not inside a
 * capture). */
LINKS_API int links_workspace_reserve(links_ctx ctx, size_t bytes);

/* ---- Serving: continuous batching of candidate batches (no counterpart in the paper;
 * the form in which the simulation path is offered as a service).  The request loop
 * runs on the GPU: a persistent cooperative kernel takes the admitted batches ("passes")
 * from a descriptor ring in device memory and runs each pass's plan build, screen,
 * valid-row compaction, emit and path normalisation between grid barriers; a host
 * thread only admits requests, copies their inputs and results, and relaunches the
 * kernel when it has exited after 2 ms without work.  While requests are in flight the
 * kernel occupies every SM. 
 * A request is a batch of `count` candidates in the layout of links_plan_build,
 * padded to the serving n_max, positions float32, all in HOST memory (pinned for
 * full overlap) that stays valid until the ticket completes.  Its outputs are
 * written to the request's host buffers before completion:
 *   valid [count] u8, lock_step [count] i16, min_disc [count] f32 (may be NULL);
 *   for the valid candidates in increasing index, up to out_capacity rows:
 *   valid_index [out_capacity] i32 (index within the request), paths
 *   [out_capacity, T, 2] f32 normalised coupler paths (may be NULL) and traj
 *   [out_capacity, n_max, T, 2] f32 (may be NULL; needs with_traj at start). */
typedef struct {
  int64_t count;
  const int32_t* n_joints;
  const uint8_t* adj;
  const int8_t* type;
  const float* pos0;
  uint8_t* valid;
  int16_t* lock_step;
  float* min_disc;
  int64_t out_capacity;
  int32_t* valid_index;
  float* paths;
  float* traj;
} links_request;

typedef struct {
  int status;        /* LINKS_OK or the failure of the request's pass */
  int64_t n_valid;   /* valid candidates (rows beyond out_capacity were not written) */
  double submit_ms;  /* steady-clock timestamps in milliseconds */
  double admit_ms;
  double done_ms;
} links_result;

/* Starts serving.  The device arena holds the candidates of every admitted request
 * (inputs, plans, flags, paths): mem_budget_bytes bounds it, and a request is admitted
 * only when its candidates fit (memory-bounded admission).  Up to max_pending requests
 * may wait for admission; T <= 256 steps; with_traj != 0 also returns trajectories.
 * The screen's lanes per mechanism and the emit's slot storage come from ctx's shape
 * table for n_max (links_set_tuning / links_autotune before this call).  Work runs on
 * the library's own streams.  LINKS_ESTATE on a device without cooperative launch. */
LINKS_API int links_serve_start(links_ctx ctx, size_t mem_budget_bytes, int max_pending, int n_max, int T,
                                int with_traj);
/* Enqueues a request (non-blocking): LINKS_EBUSY when max_pending requests already
 * wait, LINKS_ECAPACITY when the request can never fit the memory budget. */
LINKS_API int links_serve_submit(links_ctx ctx, const links_request* req, uint64_t* ticket);
/* Waits up to timeout_us for the ticket: LINKS_ETIMEDOUT if not finished (the ticket
 * stays valid); otherwise fills *res, releases the ticket and returns its status. */
LINKS_API int links_serve_poll(links_ctx ctx, uint64_t ticket, int timeout_us, links_result* res);
/* Holds (paused = 1) or resumes (0) admission of new requests; admitted work
 * continues.  For host-side fault-injection tests. */
LINKS_API int links_serve_pause(links_ctx ctx, int paused);
/* Fault injection (a host-side trigger; nothing faults the GPU): one grid barrier of the
 * next pass waits for a block that does not exist and gives up after wait_ms (1 to
 * 10000); the serving kernel then returns, and that pass's requests, with any published
 * behind it, complete with LINKS_EDEVICE (the kernel's bounded wait ran out).  Later
 * requests are served normally. */
LINKS_API int links_serve_inject_stall(links_ctx ctx, int wait_ms);
/* out[6] (host): passes published so far, launches of the serving kernel, its blocks,
 * the arena's capacity in candidates, the kernel's error word when it last returned
 * with one (1: a barrier's wait ran out, 2: the emit met a lock the screen had not
 * found, 4: a pass descriptor out of sequence), and passes finished. */
LINKS_API int links_serve_stats(links_ctx ctx, int64_t* out);
/* Finishes all submitted requests, stops the request loop and frees the arena. */
LINKS_API int links_serve_stop(links_ctx ctx);

/* Per-kernel timing for benchmarks: with enable = 1 (collection cleared), every
 * kernel the library launches on ctx is bracketed by two CUDA events on the
 * context's stream; enable = 0 stops.  Not for use inside a graph capture. */
LINKS_API int links_profile(links_ctx ctx, int enable);
/* Reads the collected timings (synchronizes the stream): up to max entries of
 * kernel name (names [max][32], NUL-terminated), total milliseconds and launch
 * count; *count receives the number of entries. */
LINKS_API int links_profile_read(links_ctx ctx, int max, char* names, double* total_ms,
                                 int64_t* launches, int* count);
/* Number of kernels the library has launched through ctx since it was created. */
LINKS_API int links_launch_count(links_ctx ctx, int64_t* out);

/* Valid-row compaction that allocates nothing (no counterpart in the paper; it
 * serves callers that cannot call cudaMalloc, e.g. code running inside a framework
 * that owns the device memory pool, or on a latency budget where an allocation may
 * block).  From valid [B] uint8 (device) it writes the indices of the nonzero
 * entries in increasing order to out_index [out_capacity] int32 (device; entries
 * beyond out_capacity are dropped) and their count to *n_out (device int32) -- the
 * same rows links_simulate writes in LINKS_OUT_VALID_ONLY mode.  Its scratch is a
 * static device array inside the library sized for B <= 4194304 (4096 x 1024
 * flags); a larger B returns LINKS_EINVAL.  It needs no context and runs on the
 * calling thread's current device and on cuda_stream (a cudaStream_t of that
 * device).  Its first call in a device's context looks up the array's device
 * address (cudaGetSymbolAddress) and caches it for that context, so make that first
 * call before any stream capture; after a device reset the new context's first call
 * looks it up again.
 * Every call on a device shares the array: calls that overlap on the GPU (other
 * streams, other threads) race and must be serialised by the caller.
 * Asynchronous. */
LINKS_API int links_compact_valid_static(const uint8_t* valid, int64_t B, int32_t* out_index,
                                         int64_t out_capacity, int32_t* n_out, void* cuda_stream);

/* ---- Kernel shapes (no counterpart in the paper; how the batched kernels are laid out
 * on the GPU).  Each context keeps a table of shapes per n_max; the keys: */
#define LINKS_TUNE_BUILDER 0      /* device plan builder: 0 default (warp-flat), 1 a thread
                                     per mechanism (n_max <= 8 only), 2 warp-flat: a lane
                                     per mechanism for the solve order, a lane per dyad for
                                     the geometry */
#define LINKS_TUNE_SCREEN_LANES 1 /* lanes per mechanism of the screen: 8 (default), 16, 32 */
#define LINKS_TUNE_SCREEN_STEPS 2 /* steps per lane of the screen: 0 by size (2 when
                                     n_max <= 9), 1, 2 (n_max <= 16 only) */
#define LINKS_TUNE_SCREEN_CTAS 3  /* CTAs per SM of the persistent screen, 0 = as many as fit */
#define LINKS_TUNE_EMIT_DWS 4     /* double-word slots of the emit: -1 by size (shared
                                     memory when n_max <= 12), 0 thread-local, 1 shared */
#define LINKS_TUNE_EMIT_CTAS 5    /* CTAs per SM of the emit, 0 = as many as fit */
#define LINKS_TUNE_SCREEN_DEFER 6 /* steps the screen's FP32 bounds leave uncertain: 0
                                     recomputed in double-word at once by their lane, 1
                                     their mechanisms left to a second, rescuing launch */

/* Autotuner: on the plan as last built, over T steps, times the screen with every shape
 * (lanes 8/16/32 x steps per lane 1/2 x CTAs per SM all/2/1 x inline or deferred
 * rescue), then the emit (shared or thread-local double-word slots x CTAs per SM
 * all/2/1) on up to 262144 packed valid rows of that screen's result (each shape once
 * to warm up, three times timed), and keeps the fastest of each in the context's table for this
 * n_max (*lanes receives the screen's lanes; may be NULL).  Each shape gives the same
 * outputs; only the time differs.  Allocates scratch and synchronizes: call it before
 * capturing a graph.  Without it the defaults above apply. */
LINKS_API int links_autotune(links_ctx ctx, links_plan plan, int T, int* lanes);

/* Sets (or reads) one key of the shape table for plans of n_max joints (2..32).
 * LINKS_EINVAL for an unknown key or a value outside the key's range for that n_max. */
LINKS_API int links_set_tuning(links_ctx ctx, int n_max, int key, int value);
LINKS_API int links_get_tuning(links_ctx ctx, int n_max, int key, int* value);
/* Writes the context's shape table to a text file (a header naming the device and its SM
 * count, then one line per n_max: n_max and the seven keys in key order), or reads one
 * back (LINKS_ESTATE if it was written on another kind of device, LINKS_EINVAL if
 * malformed or out of range; nothing is loaded then). */
LINKS_API int links_tuning_save(links_ctx ctx, const char* path);
LINKS_API int links_tuning_load(links_ctx ctx, const char* path);

/* Sets the screen's lanes per mechanism (8, 16 or 32) for plans of this n_max
 * (links_set_tuning with LINKS_TUNE_SCREEN_LANES). */
LINKS_API int links_set_screen_lanes(links_ctx ctx, int n_max, int lanes);

/* Begin / end capturing the context's stream into a reusable graph. */
LINKS_API int links_capture_begin(links_ctx ctx);
LINKS_API int links_capture_end(links_ctx ctx, links_graph* out);
LINKS_API int links_graph_launch(links_ctx ctx, links_graph graph);
LINKS_API int links_graph_free(links_graph graph);

#ifdef __cplusplus
}
#endif

#endif /* LINKS_H */
