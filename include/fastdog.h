/*
 * fastdog.h -- C ABI of the GB300 FastDOG dual hot path.
 *
 * FastDOG (Abbas & Swoboda, CVPR 2022) solves 0-1 integer linear programs
 *     min c^T x   s.t.  L_j <= a_j^T x <= U_j  (one row per constraint),  x in {0,1}^n
 * by a Lagrange decomposition with one binary decision diagram (BDD) per row
 * (Def. 1 "Binary Program", Ex. 1 "ILP", Def. 4 "BDD").  This library builds
 * the BDDs on the host, keeps the whole dual state resident on one GPU, and
 * runs every step of the method in hand-written sm_103a CUDA kernels:
 *
 *   forward / backward min-plus shortest-path sweeps     (Alg. 3, Alg. 4)
 *   min-marginal differences M_ij = m^1_ij - m^0_ij       (Eq. MM, Eq. MD, Eq. 6)
 *   parallel deferred min-marginal averaging, damping w   (Alg. 1, Eq. 5)
 *   the lower bound sum_j E^j(lambda^j)                   (Eq. D, Prop. 1)
 *   perturbation primal rounding                          (Alg. 2)
 *
 * Conventions (all entry points)
 *   - Every function returns an int status: FDOG_OK (0) or a negative code
 *     below.  No C++ exception, abort() or exit() crosses this boundary.
 *   - Pointers named host_* / plain arrays are HOST memory unless the
 *     parameter name says "dev".  Inputs are copied; the caller keeps
 *     ownership of every array it passes.  Output arrays are caller-allocated.
 *   - An instance is not thread-safe; distinct instances are independent.
 *   - A `cuda_stream` argument is a cudaStream_t passed as void*; NULL means
 *     the legacy default stream.  All device work of an instance is ordered on
 *     the stream given to fdog_build_bdds.
 *   - Floating point: sweeps, multipliers and min-marginals are FP32; lower
 *     bounds and objectives are reduced in FP64 with compensated summation,
 *     and a bound evaluated at a given state uses FP64 labels.
 */
#ifndef FASTDOG_H
#define FASTDOG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define FDOG_OK 0
#define FDOG_EINVAL (-1)        /* malformed input (CSR, sense, coefficient, parameter, NULL pointer) */
#define FDOG_ENOMEM (-2)        /* host or device allocation failed, or a row's BDD is too large */
#define FDOG_EINFEASIBLE (-3)   /* some row (after presolve) has an empty feasible set */
#define FDOG_ECUDA (-4)         /* a CUDA runtime call or kernel launch failed */
#define FDOG_ESTATE (-5)        /* call out of order (e.g. iterate before fdog_build_bdds) */
#define FDOG_ETIMEOUT (-6)      /* a bounded device-side wait expired; the context stays usable */
#define FDOG_ENOCONVERGE (-7)   /* rounding hit max_rounds; a solution is still returned, feasible=0 */
#define FDOG_EUNSUPPORTED (-8)  /* valid request this build does not handle */

/* row sense: a_j^T x <= b_j, == b_j, >= b_j */
#define FDOG_LE (-1)
#define FDOG_EQ 0
#define FDOG_GE 1

typedef struct fdog_instance fdog_instance; /* opaque, library-owned */

/*
 * Parameters.  Defaults (fdog_params_default):
 *   omega = 0.5      damping of the deferred averaging, must lie in (0, 1]
 *                    (Alg. 1 input; 0.5 in the paper's experiments, Sec. 3.3)
 *   delta = 1.0      initial perturbation strength of Alg. 2 (Sec. 6)
 *   alpha = 1.2      perturbation growth rate of Alg. 2 (Sec. 6)
 *   tol   = 1e-4     stopping rule: stop once
 *                    LB_t - LB_{t-window} <= tol * max(|LB_t|, 1)
 *                    after at least min_iters iterations (the paper stops on
 *                    the relative change of the dual objective, Sec. 3.3);
 *                    tol <= 0 disables early stopping
 *   window = 10, min_iters = 20
 *   rounding_dual_iters = 20   Alg. 1 iterations per rounding round (Alg. 2
 *                              "reoptimize"; the count is not stated)
 *   max_rounds = 200           cap on Alg. 2 rounds (termination is not
 *                              guaranteed, Sec. 4)
 *   seed = 0                   seed of the counter-based perturbation draws
 *   block_threads = 0          threads per CTA for the sweep kernels;
 *                              0 = use the built-in autotuner (it also picks
 *                              the grid mode and the dual iterations per
 *                              CUDA-graph replay, about 1 ms of device work)
 *   grid_waves = 0             sweep grid size: k > 0 = at most k waves of
 *                              resident CTAs (grid-stride loop beyond),
 *                              -1 = one CTA per group of tiles; 0 = chosen by
 *                              the autotuner (block_threads = 0) or one wave.
 *                              Results do not depend on either setting.
 *   update = 0                 dual update: 0 = parallel deferred min-marginal
 *                              averaging (Alg. 1, Eq. 5); 1 = the serial
 *                              averaging of Eq. 4 (each variable's copies
 *                              averaged at once, variables in ascending then
 *                              descending order; omega unused), run level by
 *                              level; instances with update = 1 are solved
 *                              alone (not in a batch or server)
 *   jit = 0                    shape-specialised sweep kernels, compiled with
 *                              NVRTC for BDD shapes of width <= 4 and length
 *                              <= 16: 0 = for such shapes with at least 4096
 *                              BDDs in the instance, 1 = for every such shape,
 *                              -1 = never; when NVRTC is unavailable the
 *                              instance falls back to the generic kernels
 *   fuse = 0                   deferred sums of variables whose copies all lie
 *                              in one tile of 32 BDDs are formed inside the
 *                              update sweep (same operations, same order);
 *                              -1 = leave every variable to the separate pass
 *   planner = 0                where fdog_build_bdds builds the decomposition
 *                              of an unplanned instance: 0 = on the device
 *                              when the instance allows it (else the host),
 *                              1 = on the host, 2 = on the device only
 *                              (FDOG_EUNSUPPORTED otherwise).  The device
 *                              builder takes instances whose rows need no
 *                              presolve (no row forces a variable or accepts
 *                              every assignment; rows non-empty, sorted,
 *                              without zero coefficients), with at most 1024
 *                              distinct row signatures (sense, right-hand
 *                              side, coefficient sequence), at most 4096
 *                              copies of any variable, and update = 0.  Both
 *                              builders give the same plan.
 */
typedef struct {
    double omega;
    double delta;
    double alpha;
    double tol;
    int32_t window;
    int32_t min_iters;
    int32_t rounding_dual_iters;
    int32_t max_rounds;
    uint64_t seed;
    int32_t block_threads;
    int32_t jit;
    int32_t fuse;
    int32_t grid_waves;
    int32_t update;
    int32_t planner;
    int32_t reserved[2];
} fdog_params;

/* Fill *p with the defaults above.  Returns FDOG_EINVAL if p is NULL. */
int fdog_params_default(fdog_params* p);

/*
 * Create an instance from a sparse 0-1 ILP (Ex. 1).  Row j has entries
 * col[row_ptr[j] .. row_ptr[j+1]) with integer coefficients coef[...],
 * sense[j] in {FDOG_LE, FDOG_EQ, FDOG_GE} and integer right-hand side rhs[j].
 * cost has n_vars finite entries.  All arrays are host memory and are copied.
 * Errors: FDOG_EINVAL for a negative size, a decreasing row_ptr, a column
 * out of [0, n_vars), a repeated column within a row, a bad sense, a
 * non-finite cost or invalid params; FDOG_ENOMEM.  params may be NULL
 * (defaults).  On success *out owns the instance (free with fdog_destroy).
 */
int fdog_create(int32_t n_vars, const double* cost, int32_t n_rows, const int64_t* row_ptr, const int32_t* col,
                const int32_t* coef, const int8_t* sense, const int64_t* rhs, const fdog_params* params,
                fdog_instance** out);

/*
 * Host-only planning: presolve, BDD construction and the device layout,
 * without touching a GPU.  *device_bytes (may be NULL) receives the device
 * memory fdog_build_bdds will allocate (what an admission controller needs).
 * Calling it is optional; fdog_build_bdds plans if needed.  Same errors as
 * fdog_build_bdds minus FDOG_ECUDA.
 */
int fdog_plan(fdog_instance* inst, int64_t* device_bytes);

/*
 * Introspection of a planned instance.  fdog_fixed_vars writes n_vars bytes:
 * -1 for a variable inside some BDD, 0 / 1 for a variable fixed by presolve,
 * 2 for a variable in no remaining row.  fdog_row_bdd exports the BDD of
 * original row `row` (Def. 4): *k layers over variables vars[0..k) in
 * ascending order, *n_nodes nodes, layer t = nodes [lstart[t], lstart[t+1]),
 * node 0 the root, lo/hi the 0-/1-arc successors as node indices or -1 (TOP)
 * / -2 (BOT).  Pass NULL arrays to query *k and *n_nodes; a row removed by
 * presolve gives *k = 0.  FDOG_ESTATE if not planned.
 */
int fdog_fixed_vars(fdog_instance* inst, int8_t* fixed);

/*
 * Which sweep kernels a planned instance uses: *jit_shapes distinct shapes
 * with shape-specialised kernels, covering *jit_tiles tiles of 32 BDDs;
 * *static_tiles tiles run the generic kernels; *local_vars variables have all
 * their copies in one tile, so the update sweep forms their deferred terms
 * (params.fuse); the deferred-sum kernel handles the other *work_vars
 * variables, with *work_slots copies in all.  If the specialised kernels could
 * not be compiled, `note` (capacity note_cap, may be NULL) receives the
 * reason.  Any pointer may be NULL.  FDOG_ESTATE if not planned.
 */
int fdog_kernel_plan(fdog_instance* inst, int32_t* jit_shapes, int64_t* jit_tiles, int64_t* static_tiles,
                     int64_t* local_vars, int64_t* work_vars, int64_t* work_slots, char* note, int32_t note_cap);
int fdog_row_bdd(fdog_instance* inst, int32_t row, int32_t* k, int32_t* n_nodes, int32_t* vars, int32_t* lstart,
                 int32_t* lo, int32_t* hi);

/*
 * How the plan was built: *on_device = 1 if by the device builder (see
 * params.planner), *seconds = wall time of building the decomposition (BDDs,
 * layout, slot lists; without the NVRTC compile).  Either pointer may be
 * NULL.  FDOG_ESTATE if not planned.
 */
int fdog_plan_stats(fdog_instance* inst, int32_t* on_device, double* seconds);

/*
 * Fingerprints of a planned instance's decomposition, one FNV-1a 64-bit
 * digest per part, written to digest[0..FDOG_PLAN_DIGESTS):
 *   0 presolve (fixed flags, constants)   1 shapes and templates
 *   2 tiles and class ranges              3 slot variables (var)
 *   4 per-variable slot lists             5 tile-local patterns and entries
 *   6 deferred-sum buckets (work, wpos)   7 BDD <-> row maps
 *   8 counts (BDDs, slots, nodes, local and work variables)
 * Two plans with equal digests lay out every device array identically.  For
 * a plan built on the device the arrays are read back once (host copy kept).
 * FDOG_ESTATE if not planned; FDOG_ECUDA if the read-back fails.
 */
#define FDOG_PLAN_DIGESTS 9
int fdog_plan_digest(fdog_instance* inst, uint64_t* digest);

/*
 * Long-row splitting (the paper's conclusion names long rows as future
 * work): a transformation of an ILP given in the fdog_create form, applied by
 * the caller before fdog_create.  Every row sum_{i in I} x_i <= 1 or = 1
 * (all coefficients 1, right-hand side 1) with |I| > max_len becomes a chain
 * of rows of at most max_len variables joined by new binary variables
 * y_1 .. y_{m-1} (numbered from n_vars on, cost 0 for the caller to append):
 *   sum_{P_1} x - y_1 = 0,  sum_{P_j} x + y_{j-1} - y_j = 0,
 *   sum_{P_m} x + y_{m-1} <= 1 (= 1),
 * with |P_1| = max_len - 1, |P_j| = max_len - 2 and |P_m| <= max_len - 1, the
 * entries of P in the row's order.  Pieces share one binary variable each, so
 * the split rows have the same convex hull over x as the original row and the
 * decomposition the same optimal bound, with BDDs of at most max_len layers.
 * Other rows are copied unchanged; pieces replace their row in place, and
 * out_row_origin (may be NULL) gives each new row's original row.
 * Size query: out_row_ptr NULL writes *out_n_vars, *out_n_rows, *out_nnz;
 * otherwise those give the capacities of the caller's arrays
 * (out_row_ptr[*out_n_rows + 1], out_col / out_coef[*out_nnz],
 * out_sense / out_rhs / out_row_origin[*out_n_rows]) and receive the sizes.
 * Errors: FDOG_EINVAL (max_len < 3, malformed CSR, NULL pointers, capacity
 * too small), FDOG_EUNSUPPORTED (more than 2^31 - 1 variables or rows).
 */
int fdog_split_rows(int32_t n_vars, int32_t n_rows, const int64_t* row_ptr, const int32_t* col, const int32_t* coef,
                    const int8_t* sense, const int64_t* rhs, int32_t max_len, int32_t* out_n_vars,
                    int32_t* out_n_rows, int64_t* out_nnz, int64_t* out_row_ptr, int32_t* out_col,
                    int32_t* out_coef, int8_t* out_sense, int64_t* out_rhs, int32_t* out_row_origin);

/*
 * Build the decomposition and upload it to `device` on `cuda_stream`:
 * presolve (fix variables a row forces, drop rows every assignment
 * satisfies), one reduced ordered BDD per remaining row over its variables in
 * ascending index order (Def. 4; arcs leaving layer i carry lambda_i as in
 * Fig. 3), the node layout, and the initial multipliers
 * lambda^j_i = c_i / |J_i| with M-bar = 0 (Alg. 1 text).
 * The decomposition of an unplanned instance is built on the device or the
 * host as params.planner says.
 * Errors: FDOG_EINFEASIBLE (a row cannot be satisfied), FDOG_ENOMEM (host or
 * device memory, or a row whose BDD exceeds the node limit), FDOG_ECUDA,
 * FDOG_EUNSUPPORTED (a BDD wider or longer than the sweep kernels take;
 * planner = 2 and an instance the device builder does not take),
 * FDOG_ESTATE if already built.  After fdog_release the instance may be
 * built again (on any device and stream); its plan is reused.
 */
int fdog_build_bdds(fdog_instance* inst, int32_t device, void* cuda_stream);

/*
 * Free the instance's device memory (no counterpart in the paper: memory
 * management for callers that keep many instances).  The plan, the last
 * rounded solution and its objective stay readable on the host; the dual
 * state is dropped.  Waits for the instance's stream first.  FDOG_OK also
 * when nothing is resident.
 */
int fdog_release(fdog_instance* inst);

/*
 * Host memory (no counterpart in the paper).  Large host arrays that
 * instances free (their copies of the ILP, host plans) are kept in a
 * process-wide cache, at most 2 GiB, and reused by later instances of the
 * same sizes, whose pages are then already mapped.  This call frees every
 * cached buffer; *bytes_freed (may be NULL) receives their total size.
 * Thread-safe; buffers in use by live instances are not affected.
 */
int fdog_host_cache_release(int64_t* bytes_freed);

/*
 * Re-initialise the dual state on the device: lambda^j_i = c_i / |J_i|,
 * M-bar = 0, iteration counter and stopping history cleared (Alg. 1
 * initialisation).  The decomposition stays resident.
 */
int fdog_reset_dual(fdog_instance* inst);

/*
 * Run up to k iterations of Alg. 1 (one ascending and one descending pass
 * each, Eq. 5 updates, deferred sums refreshed after every pass), stopping
 * early when the stopping rule of fdog_params holds.  The deferred
 * differences of the last pass stay pending (see fdog_lower_bound).
 * *iters_done (may be NULL) receives the iterations run by this call and *lb
 * (may be NULL) the running lower bound after the last one.  Blocks until the
 * device work is done.  Errors: FDOG_ESTATE (not built), FDOG_EINVAL (k < 0),
 * FDOG_ECUDA.
 */
int fdog_dual_iterate(fdog_instance* inst, int32_t k, int32_t* iters_done, double* lb);

/*
 * Final loop of Alg. 1: add the pending deferred differences back,
 * lambda^j_i += omega / |J_i| sum_k Mbar_ik, so that sum_j lambda^j_i = c_i
 * again (dual feasibility, Prop. 1).  No-op if nothing is pending.  A later
 * fdog_dual_iterate restarts Alg. 1 from M-bar = 0.
 */
int fdog_finalize(fdog_instance* inst);

/*
 * Lower bounds at the current state, both valid for the ILP (Prop. 1):
 *   *lb_running  = sum_j E^j of the lifted multipliers (the bound the
 *                  iterations report; non-decreasing),
 *   *lb_feasible = sum_j E^j(lambda^j) after adding the pending deferred
 *                  differences back (Alg. 1, last loop), i.e. at dual-feasible
 *                  multipliers with sum_j lambda^j_i = c_i.
 * Both include the constant of variables fixed by presolve or in no row.
 * *lb_feasible (and *lb_running when no iteration has run since the state was
 * last set) is evaluated with FP64 shortest-path labels over the FP32
 * multipliers and summed with FP64 Neumaier in a fixed order; *lb_running
 * after iterations is the bound the last iteration reduced (FP32 per-BDD
 * energies, compensated sums).  Either pointer may be NULL.  Does not modify
 * the state.
 */
int fdog_lower_bound(fdog_instance* inst, double* lb_running, double* lb_feasible);

/*
 * Min-marginals (Eq. MM) of every (row, variable) slot at the current
 * multipliers lambda (pending deferred differences NOT added), computed on
 * the GPU by Eq. 6.  If var == NULL the call only stores the slot count in
 * *n_slots.  Otherwise *n_slots must hold the capacity of the four arrays;
 * slot s is (row[s], var[s]) with min-marginals m0[s], m1[s]; rows are the
 * caller's original row indices.  FDOG_EINVAL if the capacity is too small.
 */
int fdog_min_marginals(fdog_instance* inst, int64_t* n_slots, int32_t* var, int32_t* row, float* m0, float* m1);

/*
 * Current multipliers lambda^j_i of every slot (same slot order and size
 * query convention as fdog_min_marginals).  lambda may be NULL.
 */
int fdog_multipliers(fdog_instance* inst, int64_t* n_slots, int32_t* var, int32_t* row, float* lambda);

/*
 * Perturbation primal rounding (Alg. 2): add the pending deferred
 * differences back, compute all M_ij, and while some variable's M_ij do not
 * all share one strict sign, perturb every variable by the four cases of
 * Alg. 2: +delta / -delta where all M_ij are positive / negative, r * delta
 * where all are zero, sign(sum_j M_ij) |r| delta otherwise, with r uniform in
 * [-delta, delta) from u = SplitMix64(seed ^ round<<32 ^ i) as
 * r = delta (2u - 1); then grow delta by alpha, re-run rounding_dual_iters
 * iterations of Alg. 1 and the add-back, and recompute M.  At agreement
 * x_i = [M_ij < 0].
 * *rounds_used (may be NULL) receives the number of perturbation rounds.
 * Returns FDOG_ENOCONVERGE after max_rounds rounds without agreement (the
 * solution is then x_i = [sum_j M_ij < 0], possibly infeasible).
 * The multipliers are left perturbed (Alg. 2 does not keep them feasible).
 */
int fdog_primal_round(fdog_instance* inst, int32_t* rounds_used);

/*
 * The last rounded solution: x (n_vars bytes, may be NULL), its objective
 * c^T x summed in FP64 (may be NULL), and *feasible = 1 iff x satisfies every
 * row exactly (integer check on the host; may be NULL).
 * FDOG_ESTATE if fdog_primal_round has not run.
 */
int fdog_solution(fdog_instance* inst, uint8_t* x, double* objective, int32_t* feasible);

/*
 * Checkpoint: the complete resumable dual state (multipliers, deferred sums,
 * per-variable targets, iteration count, stopping history).  If buf is NULL,
 * *bytes receives the size.  fdog_import_state restores a state exported
 * from an instance built from the same ILP and parameters; a resumed run is
 * bit-identical to an uninterrupted one.  FDOG_EINVAL on a size or
 * signature mismatch.
 */
int fdog_export_state(fdog_instance* inst, void* buf, size_t* bytes);
int fdog_import_state(fdog_instance* inst, const void* buf, size_t bytes);

/*
 * Sizes of the built decomposition (any pointer may be NULL): variables,
 * BDDs, slots (sum_j |I_j|), BDD nodes, and device bytes held.
 */
int fdog_info(fdog_instance* inst, int64_t* n_vars, int64_t* n_bdds, int64_t* n_slots, int64_t* n_nodes,
              int64_t* device_bytes);

/*
 * Bytes the library has copied host-to-device and device-to-host for this
 * instance since it was created (uploads, control-block reads, results).
 */
int fdog_transfer_bytes(fdog_instance* inst, int64_t* h2d, int64_t* d2h);

/*
 * Kernel timing.  While profiling is on, every update-pass sweep launch (the
 * ascending / descending passes of Alg. 1) and every deferred-sum step is
 * bracketed by CUDA events on the stream it runs on (iteration graphs are
 * not used meanwhile).  fdog_profile_read synchronises the stream and
 * returns, since the last read, the launches and summed device milliseconds
 * of the sweeps of each pass's dominant kernel class (the one with the most
 * tile-layers) and of the deferred-sum steps, plus *kernel_launches = all
 * kernel launches of the instance since it was built (always counted).  Any
 * output pointer may be NULL.
 */
int fdog_set_profiling(fdog_instance* inst, int32_t on);
int fdog_profile_read(fdog_instance* inst, int64_t* sweep_launches, double* sweep_ms, int64_t* reduce_launches,
                      double* reduce_ms, int64_t* kernel_launches);

/*
 * Ragged batching.  A batch runs several built instances (same device) as one
 * flat index space of BDD tiles and variables: every kernel launch covers all
 * members, so many small instances fill the GPU as one large one would.  Each
 * member follows its own schedule -- Alg. 1 until its stopping rule (or
 * max_iters iterations), then Alg. 2 -- and gets exactly the results it would
 * get alone (all reductions are per instance in a fixed order).  Iterations
 * run as CUDA-graph replays on cuda_stream when it is not NULL; the sweep
 * kernels' warps per block, grid mode and iterations per replay are
 * autotuned at creation when the first member's params.block_threads is 0.  Members stay owned by the caller and must
 * outlive the batch; an instance may belong to one batch call at a time.
 *
 * fdog_batch_solve: Alg. 1 then Alg. 2 for every member from its current
 * state; per member (arrays of n entries, each may be NULL) the dual
 * iterations run, the rounding rounds used and FDOG_OK / FDOG_ENOCONVERGE.
 * Solutions are then available through fdog_solution on each member.
 * fdog_batch_info: the chosen warps per block, iterations per graph replay,
 * and the batch's kernel launches so far.
 */
typedef struct fdog_batch fdog_batch;
int fdog_batch_create(fdog_instance* const* insts, int32_t n, void* cuda_stream, fdog_batch** out);
/*
 * fdog_batch_set_persistent (no counterpart in the paper: a way to run the
 * batch): on = 1 runs each chunk of dual iterations of fdog_batch_solve as
 * one persistent cooperative kernel whose blocks stay resident and pass the
 * device-wide barriers of Alg. 1 (after each pass, after the deferred sums,
 * after the bound) through a grid barrier of their own, instead of graph
 * replays of per-pass kernels; on = 0 returns to the graph replays.  Results
 * are the same bit for bit.  A block that waits at a barrier longer than
 * barrier_wait_s seconds (0: 1 s) gives up: every block leaves the kernel,
 * the members' control blocks carry the error and fdog_batch_solve returns
 * FDOG_ETIMEOUT (the context stays usable; fdog_reset_dual clears the
 * members).  Takes batches whose BDDs all have width <= 2 and run on the
 * generic kernels (params.jit = -1 on every member): FDOG_EUNSUPPORTED
 * otherwise.  FDOG_EINVAL for a bad flag or a negative wait.
 */
int fdog_batch_set_persistent(fdog_batch* batch, int32_t on, double barrier_wait_s);
int fdog_batch_solve(fdog_batch* batch, int32_t max_iters, int32_t* iters, int32_t* rounds, int32_t* status);
int fdog_batch_info(fdog_batch* batch, int32_t* warps_per_block, int32_t* chunk, int64_t* kernel_launches);
const char* fdog_batch_last_error(const fdog_batch* batch);
void fdog_batch_destroy(fdog_batch* batch);

/*
 * Continuous-batching server.  A worker thread on `device` keeps every
 * admitted instance's BDDs and dual state resident and advances all of them
 * together: each scheduling step runs a chunk of dual iterations for the
 * instances still iterating and the rounding tests / perturbations of the
 * others, so requests that arrive while others are on the GPU join the
 * running set as soon as a slot (max_active) and HBM (hbm_budget bytes) are
 * free, in arrival order.  An instance is
 * retired when its stopping rule (tol, window, min_iters, or max_iters
 * iterations) has fired and rounding has agreed (or hit max_rounds); its
 * device memory is then freed and its solution kept on the host.  Results
 * equal those of solving each instance alone.
 *
 * fdog_server_submit: `inst` must be created and not built; ownership moves
 * to the server until fdog_server_take.  *ticket identifies the request.  An
 * unplanned instance is only queued, with an upper bound of the device
 * memory it may need (from its sizes); at admission the worker builds its
 * decomposition on the device (the host builder for instances the device
 * builder does not take, see params.planner) and the reservation becomes
 * the memory the instance holds.  Planning errors then arrive as the
 * request's status (fdog_server_poll).  An instance already planned
 * (fdog_plan) or with planner = 1 is planned here, in the caller's thread,
 * and its errors are returned here.
 * fdog_server_poll: *state 0 queued, 1 resident, 2 done; *status FDOG_OK /
 * FDOG_ENOCONVERGE / error of the request; *lb the running bound at
 * retirement; *latency_s submit-to-done time (or time so far).
 * fdog_server_wait: blocks until the request is done or timeout_s passes
 * (FDOG_ETIMEOUT).
 * fdog_server_take: hands a done instance back (fdog_solution works on it;
 * free it with fdog_destroy).
 * fdog_server_stats: queued and resident requests, completed ones, HBM in
 * use, seconds the worker spent on device work, kernel launches.
 * fdog_server_destroy: stops the worker and destroys instances not taken.
 */
typedef struct fdog_server fdog_server;
int fdog_server_create(int32_t device, int64_t hbm_budget, int32_t max_active, int32_t max_iters, fdog_server** out);
int fdog_server_submit(fdog_server* srv, fdog_instance* inst, uint64_t* ticket);
int fdog_server_poll(fdog_server* srv, uint64_t ticket, int32_t* state, int32_t* status, double* lb,
                     double* latency_s);
int fdog_server_wait(fdog_server* srv, uint64_t ticket, double timeout_s);
int fdog_server_take(fdog_server* srv, uint64_t ticket, fdog_instance** out);
int fdog_server_stats(fdog_server* srv, int64_t* queued, int64_t* resident, int64_t* completed, int64_t* hbm_used,
                      double* busy_s, int64_t* kernel_launches);
const char* fdog_server_last_error(const fdog_server* srv);
void fdog_server_destroy(fdog_server* srv);

/*
 * One instance split over several GPUs (the paper's conclusion names
 * multi-GPU support as future work).  Within one pass of Alg. 1 the BDDs are
 * independent (Eq. 5 reads only a BDD's own multipliers and the deferred
 * terms of the previous pass); they are coupled only through the deferred
 * term T_i = (c_i - sum_j lambda^j_i) / |J_i| (Prop. 1), a sum over every copy
 * of variable i.  So the rows are split into shards, each an ordinary
 * instance of its own rows (one process and one GPU per shard), and once per
 * pass the shards all-reduce one float per variable whose copies lie in
 * several shards, and once per iteration the lower bound.  The all-reduce is
 * the caller's (NCCL or any other); these calls produce and consume the
 * per-shard sums on the instance's stream.  Rounding (Alg. 2) is not run on
 * shards.
 *
 * fdog_shard_plan (host only): splits rows 0..n_rows-1 of an ILP in the
 * fdog_create form into n_shards blocks with about equal numbers of non-zero
 * entries, contiguous in the order of each row's smallest variable (ties by
 * row index), so that rows over nearby variables share a shard:
 * row_shard[j] (n_rows), copies[i] = |J_i|, the rows
 * with a non-zero coefficient on variable i (n_vars), shared[i] = 1 when
 * rows of more than one shard hold i (n_vars).  coef may be NULL (every entry
 * counts).  FDOG_EINVAL on a malformed CSR or n_shards < 1.
 *
 * fdog_shard_setup: marks a created, unplanned instance as one shard.  Its
 * ILP is the whole ILP's variables (same n_vars) with this shard's rows; a
 * variable with no row in the shard should carry cost 0 there (its cost
 * belongs to the shards that hold it, or to one shard if no row holds it).
 * shared / copies are the arrays fdog_shard_plan wrote.  The plan is built on
 * the host and must need no presolve (FDOG_EUNSUPPORTED otherwise, at build).
 * FDOG_ESTATE if already planned; FDOG_EUNSUPPORTED for update = 1.
 * fdog_shard_info: *n_shared = the number of shared variables of the split
 * instance (sum of shared[]), the length of the exchange buffer, the same on
 * every shard; entry k belongs to the k-th shared variable in ascending
 * index order.  Plans the instance if needed.
 *
 * One iteration of Alg. 1 over all shards, on every shard:
 *   fdog_shard_pass(inst, 0, dev_sums)   ascending pass over the shard's BDDs,
 *                                        deferred terms of its unshared
 *                                        variables, dev_sums[k] = this shard's
 *                                        sum of lambda over the k-th shared
 *                                        variable's copies, 0 where it holds
 *                                        none (device memory of n_shared
 *                                        floats, caller-owned)
 *   all-reduce (sum) dev_sums over the shards
 *   fdog_shard_apply(inst, dev_sums)     T_i of the shared variables
 *   fdog_shard_pass(inst, 1, dev_sums)   the same for the descending pass; it
 *                                        also reduces the shard's part of the
 *                                        lower bound
 *   all-reduce dev_sums, fdog_shard_apply
 *   fdog_shard_bound(inst, &part)        (waits) this shard's part: the lifted
 *                                        energies of its BDDs plus its
 *                                        presolve constant
 *   all-reduce (sum) part
 *   fdog_shard_commit(inst, lb, &stop)   (waits) records the iteration's bound
 *                                        and runs the stopping rule; *stop = 1
 *                                        when it fired (every shard given the
 *                                        same bound decides the same)
 * Work is queued on the instance's stream; an all-reduce must be ordered
 * after the pass and before the apply on that stream.  fdog_finalize,
 * fdog_lower_bound, fdog_min_marginals and fdog_multipliers work on a shard
 * and describe its own BDDs: its bounds are this shard's part, except
 * lb_running after iterations, which is the last committed bound of the
 * whole instance.
 * fdog_dual_iterate returns FDOG_ESTATE on a shard; fdog_primal_round,
 * batches and servers refuse shards (FDOG_EUNSUPPORTED).  Errors:
 * FDOG_EINVAL (NULL buffer with shared variables, bad direction),
 * FDOG_ESTATE (not a shard, not built, no descending pass before
 * fdog_shard_bound), FDOG_ECUDA.
 */
int fdog_shard_plan(int32_t n_vars, int32_t n_rows, const int64_t* row_ptr, const int32_t* col, const int32_t* coef,
                    int32_t n_shards, int32_t* row_shard, int32_t* copies, uint8_t* shared);
int fdog_shard_setup(fdog_instance* inst, const uint8_t* shared, const int32_t* copies);
int fdog_shard_info(fdog_instance* inst, int32_t* n_shared);
int fdog_shard_pass(fdog_instance* inst, int32_t descending, float* dev_sums);
int fdog_shard_apply(fdog_instance* inst, const float* dev_sums);
int fdog_shard_bound(fdog_instance* inst, double* lb_part);
int fdog_shard_commit(fdog_instance* inst, double lb, int32_t* stop);

/*
 * Allocation-free lower-bound reduction (the paper has no counterpart: this
 * serves callers that cannot allocate device memory -- plug-ins whose host
 * framework owns every device allocation through its own pool, and real-time
 * loops that forbid allocation after start-up).
 * Writes to dev_out[0] the deterministic FP64 compensated sum
 * constant + sum_{t < n} dev_values[t] -- e.g. per-subproblem energies E_j, so
 * that the result is the bound sum_j E^j of Eq. D -- with the same two-stage
 * compensated reduction as the library's own bound kernels: per-block
 * partials (256 values per block), then a last-block Neumaier sum of them.
 * dev_values (n doubles) and dev_out (one double) are device memory owned by
 * the caller; the call allocates nothing: its scratch is a static device
 * array of 256 KiB that every GPU loading this library holds until the
 * process exits.  n = 0 writes `constant`.
 * n may be at most 8,388,608 (FDOG_EINVAL beyond, or for negative n or NULL
 * pointers).  The first call on a device looks up that array's device address
 * with the device current, and so does the first call after cudaDeviceReset
 * (the address is cached per device and context); make those calls before
 * any stream capture.
 * Work is queued on cuda_stream (NULL: legacy default stream); the call does
 * not wait for it.  All calls share the one scratch array, so calls whose
 * kernels overlap on the GPU (different streams, or several host threads)
 * race: serialise them.  Errors: FDOG_EINVAL, FDOG_ECUDA.
 */
int fdog_bound_reduce_noalloc(const double* dev_values, int64_t n, double constant, double* dev_out,
                              void* cuda_stream);

/*
 * Human-readable detail of the last error status returned for this instance
 * (empty if none).  The pointer stays valid until the next call on inst.
 */
const char* fdog_last_error(const fdog_instance* inst);

/* Free the instance and its device memory.  NULL is accepted. */
void fdog_destroy(fdog_instance* inst);

/* Static text for a status code. */
const char* fdog_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* FASTDOG_H */
