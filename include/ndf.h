/*
 * ndf.h -- C ABI of libndf.so, the GB300 (sm_103a) dependence-volume library.
 *
 * The library computes, for one selected reference vertex and every vertex of
 * a 3-D grid, the statistical dependence across an M-member ensemble
 * (Sec. 3: R_mu,nu(p_mu, p_nu) = rho(e^mu(p_mu), e^nu(p_nu)), one 3-D slice of
 * the dependence field at a time), with two measures:
 *   - Pearson's r (Sec. 3.1, Eq. 1);
 *   - mutual information (Sec. 3.2, Eq. 2) by the Kraskov-Stoegbauer-
 *     Grassberger k-nearest-neighbour estimator, algorithm 1 (the estimator
 *     cited in Sec. 3.2 and timed in Sec. 6.2, Table 1).
 *
 * Conventions shared by every call:
 *   - Every call returns an ndf_status; nothing throws across the ABI.  On a
 *     failure, ndf_last_error(ctx) holds a one-line description.
 *   - Ensemble layout: float field[M][Z][Y][X], member-major; the flat vertex
 *     index is v = (z*Y + y)*X + x, element offset m*N + v with N = X*Y*Z.
 *   - Pointers may be host or device memory; the library detects which with
 *     cudaPointerGetAttributes.  Inputs are copied, never retained.  Output
 *     buffers are owned by the caller.
 *   - Work runs on the context's stream.  With device outputs a call returns
 *     once the work is enqueued; with host outputs it returns after the copy
 *     to the host has completed.  Argument errors are detected on the host
 *     and returned before anything is enqueued.
 *   - A context is not thread safe: use one context per host thread.
 */
#ifndef NDF_H
#define NDF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ndf_ctx ndf_ctx; /* opaque; owns all device memory it allocates */

/* Arithmetic of the batched Pearson volumes. */
typedef enum {
    NDF_PREC_FP32 = 0,   /* exact FP32 CUDA-core volumes, one per reference */
    NDF_PREC_BF16X3 = 1, /* tensor cores, z = hi + lo in BF16, 3 products, FP32 accumulate */
    NDF_PREC_TF32 = 2    /* tensor cores, z rounded to TF32, FP32 accumulate */
} ndf_precision;

typedef enum {
    NDF_OK = 0,
    NDF_ERR_ARG = -1,     /* invalid argument (sizes, indices, k, null pointers) */
    NDF_ERR_OOM = -2,     /* device or host allocation failed */
    NDF_ERR_CUDA = -3,    /* a CUDA runtime call or kernel launch failed */
    NDF_ERR_TIMEOUT = -4, /* a bounded device-side wait gave up */
    NDF_ERR_STATE = -5,   /* call not valid in the current state (e.g. freed field) */
    NDF_ERR_IO = -6       /* file read/write failed */
} ndf_status;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to run on (e.g. PyTorch's current stream) or NULL for a context-owned
 * non-blocking stream.  Fails with NDF_ERR_CUDA when the device is missing or
 * is not compute capability 10.3. */
ndf_status ndf_create(ndf_ctx** out, int device, void* cuda_stream);

/* Free every device buffer of the context (fields, scratch) and the context. */
void ndf_destroy(ndf_ctx* ctx);

/* Static description of a status code. */
const char* ndf_status_str(int status);

/* Detail of the last failure on this context (context-owned string). */
const char* ndf_last_error(const ndf_ctx* ctx);

/* Switch the stream later calls run on (NULL: the context's own stream). */
ndf_status ndf_set_stream(ndf_ctx* ctx, void* cuda_stream);

/* Block until all work enqueued by this context has finished. */
ndf_status ndf_synchronize(ndf_ctx* ctx);

/* Number of CUDA kernels this context has launched so far. */
uint64_t ndf_launch_count(const ndf_ctx* ctx);

/* Flat vertex index (z*Y + y)*X + x, or -1 when a coordinate is out of range. */
int64_t ndf_index(int64_t x, int64_t y, int64_t z, int64_t X, int64_t Y, int64_t Z);

/* ---- ensembles (Sec. 3: E = {E_i}, member samples e(p) of length M) ------ */

/* Copy field[M][Z][Y][X] (host or device) into context-owned device memory and
 * compute the per-vertex statistics used by Eq. 1: the FP64 mean mu_v and
 * 1/sqrt(S_v) with S_v = sum_m (e_m(v) - mu_v)^2 (FP32 sums over blocks of
 * at most 32 members, centred on the column's median member for M <= 1024 and on
 * its FP32 mean above, the blocks combined in double-float or FP64; relative
 * error of order 1e-7).  For M <= 4096 every vertex column is also sorted into a
 * second M*N*4-byte buffer (the KSG marginal counts of Algorithm 1 search it).
 * A host field is copied in vertex ranges on an internal stream, the statistics
 * and sorts of each range following on the context's stream; a device field is
 * read in place by one kernel that writes the copy, the statistics and the sorted
 * columns (M <= 1024; a contiguous copy first above that); its writes on other
 * streams must be complete before the call.  The call returns when all is done.  Requires M >= 2 and finite values (NDF_ERR_ARG otherwise; the check
 * reads the copied field).  Writes the new field's id. */
ndf_status ndf_load_ensemble(ndf_ctx* ctx, const float* field, int64_t M, int64_t Z, int64_t Y,
                             int64_t X, int* field_id_out);

/* Release a field; its id becomes invalid (NDF_ERR_STATE).  The field's device
 * buffers stay with the context (at most 8 of them, the oldest freed beyond
 * that) and a later ndf_load_ensemble of the same M*N reuses them instead of
 * allocating; ndf_trim_cache or ndf_destroy returns them to the device. */
ndf_status ndf_free_ensemble(ndf_ctx* ctx, int field_id);

/* Load an ensemble (as ndf_load_ensemble) and compute one reference vertex's
 * Pearson volume (Sec. 3.1) and KSG-MI volume (algorithm 1, Sec. 3.2) with the
 * upload pipelined against the computation: a host field is copied in vertex
 * ranges (the reference's range first) on the context's copy stream, and each
 * range's statistics, column sort and KSG search run on the context's stream as
 * soon as it has arrived (a device field is read in place, range by range, the
 * sorts writing the copy); Pearson follows the last range.  The same kernels as
 * ndf_load_ensemble + ndf_pearson + ndf_mi_ksg, so the same results.  Outputs
 * (host or device, N floats each) may be NULL to skip that measure.  The field
 * stays loaded (*field_id_out).  Errors as ndf_load_ensemble, ndf_pearson and
 * ndf_mi_ksg; non-finite input is reported after the pipeline drained
 * (NDF_ERR_ARG, nothing stays loaded). */
ndf_status ndf_load_and_compute(ndf_ctx* ctx, const float* field, int64_t M, int64_t Z, int64_t Y,
                                int64_t X, int64_t ref_idx, int k, float* pearson_out,
                                float* mi_out, int* field_id_out);

/* Free every device buffer the context keeps from released fields (synchronizes
 * the context's stream first). */
ndf_status ndf_trim_cache(ndf_ctx* ctx);

/* Test hook for failure detection: runs one kernel whose mbarrier wait is never
 * completed, so the library's bounded wait gives up (after about one second),
 * sets the device status word and returns.  The call synchronizes and returns
 * what the next host check reports: NDF_ERR_TIMEOUT when the path works.  The
 * context stays usable; the status word is cleared by the check. */
ndf_status ndf_selftest_timeout(ndf_ctx* ctx);

/* Shape of a loaded field (any output pointer may be NULL). */
ndf_status ndf_field_shape(const ndf_ctx* ctx, int field_id, int64_t* M, int64_t* Z, int64_t* Y,
                           int64_t* X);

/* Copy the per-vertex statistics (N doubles each, host or device; either may
 * be NULL): mean_out = mu_v, inv_norm_out = 1/sqrt(S_v) (0 where S_v = 0). */
ndf_status ndf_field_stats(ndf_ctx* ctx, int field_id, double* mean_out, double* inv_norm_out);

/* Copy the sorted member columns of vertices [v_begin, v_end) into out (host or
 * device, caller-owned): out[m * (v_end - v_begin) + (v - v_begin)] is the m-th
 * smallest of e_1(v) .. e_M(v), the order the KSG marginal counts of Algorithm 1
 * search.  Needs 0 <= v_begin <= v_end <= N (NDF_ERR_ARG otherwise) and a field
 * with M <= 4096, whose sorted copy is made on load (NDF_ERR_STATE above that).
 * Synchronizes the context's stream. */
ndf_status ndf_field_sorted_columns(ndf_ctx* ctx, int field_id, int64_t v_begin, int64_t v_end,
                                    float* out);

/* ---- exact estimators ---------------------------------------------------- */

/* Errors of every volume call in this section (and of the debug hooks):
 *   NDF_ERR_ARG     a field id that was never issued, fields of different
 *                   shape, a reference (or query) index outside [0, N), a null
 *                   output, R < 1 or a null index list (batches), an unknown
 *                   precision; for KSG also k outside [1, M), k > 16 or M > 4096;
 *   NDF_ERR_STATE   a field that has been freed;
 *   NDF_ERR_OOM     scratch or output staging could not be allocated;
 *   NDF_ERR_CUDA    a launch or copy failed;
 *   NDF_ERR_TIMEOUT a bounded device wait gave up (reported by the next host
 *                   check: a call with host outputs, or ndf_synchronize).
 * Argument errors leave the outputs untouched. */

/* Pearson volume (Sec. 3.1, Eq. 1): out[v] = r(e^ref(p_ref), e^query(v)) for
 * all N vertices v of the query field, FP32, clamped to [-1, 1]; 0 where
 * either sample has zero variance.  ref_field may equal query_field (the
 * self-correlation slice S_mu(p_ref, .), Sec. 3).  Fields must have the same
 * shape.  ref_idx is a flat vertex index in [0, N).  out: N floats. */
ndf_status ndf_pearson(ndf_ctx* ctx, int ref_field, int query_field, int64_t ref_idx, float* out);

/* R Pearson volumes in one call (Sec. 3.1, Eq. 1; the slices R(p_ref_i, .) of
 * Sec. 3 for R reference vertices): out[i*N + v] = r(ref_idx[i], v), FP32,
 * clamped to [-1, 1].  ref_idx: R host indices in [0, N).  out: R*N floats,
 * host or device.  With NDF_PREC_TF32 / NDF_PREC_BF16X3 the volumes are one
 * GEMM of standardised data, z = (e - mu) / sqrt(S), on the tensor cores
 * (chunks of 256 references); the standardised copy of each field is built on
 * the first such call and kept with the field (4 bytes per member and vertex,
 * members padded to a multiple of 64).  NDF_PREC_FP32 runs the exact
 * single-reference kernel R times. */
ndf_status ndf_pearson_batch(ndf_ctx* ctx, int ref_field, int query_field, const int64_t* ref_idx,
                             int R, ndf_precision prec, float* out);

/* KSG mutual-information volume (Sec. 3.2, Eq. 2; estimator of Sec. 6.2):
 * out[v] = I(e^ref(p_ref); e^query(v)) in nats, FP32, for all N vertices.
 * Algorithm 1: joint max-norm distances in FP32, eps_i = distance to the k-th
 * nearest other member, n_x / n_y = members strictly closer than eps_i in each
 * marginal (self excluded), I = psi(k) + psi(M) - <psi(n_x+1) + psi(n_y+1)>,
 * the digamma sum in FP64.  Raw values, no jitter, no clamping of negative
 * estimates.  Requires 1 <= k < M, k <= 16 and M <= 4096. */
ndf_status ndf_mi_ksg(ndf_ctx* ctx, int ref_field, int query_field, int64_t ref_idx, int k,
                      float* out);

/* KSG algorithm 2 of the same article (Sec. 3.2 cites it; row f1): per member,
 * the neighbour set S_i = {j != i : d_ij <= eps_i} (the k nearest; every member
 * tied at eps_i belongs to it), its marginal extents ex_i / ey_i (largest |dx| /
 * |dy| over S_i, FP32), non-strict counts n_x = #{j != i : |x_i - x_j| <= ex_i},
 * n_y likewise, and I2 = psi(k) - 1/k + psi(M) - <psi(n_x) + psi(n_y)> (FP64
 * sum).  Same search (ndf_set_ksg_algorithm), same limits and output as
 * ndf_mi_ksg. */
ndf_status ndf_mi_ksg2(ndf_ctx* ctx, int ref_field, int query_field, int64_t ref_idx, int k,
                       float* out);

/* KSG search used by ndf_mi_ksg, ndf_mi_ksg2, ndf_mi_ksg_batch, the debug hooks
 * and ndf_train's MI targets.  All give identical results (same FP32 distances,
 * same counts):
 *   NDF_KSG_PRUNED  two warps per (reference, vertex) pair; members in
 *                   order of the reference value, each side of a member's
 *                   outward scan stopped at the first x-gap that reaches its
 *                   current k-th distance (exact pruning);
 *   NDF_KSG_BLOCK   two warps per pair; members cut into blocks of 64 x-ranks,
 *                   sorted by the query value inside each block; a member scans
 *                   blocks outward in x and, inside a block, outward in y, both
 *                   stopped by its current k-th distance (exact pruning).
 *                   Algorithm 1 only: ndf_mi_ksg2 runs NDF_KSG_PRUNED instead;
 *   NDF_KSG_LANES   (default) the same two-level search scheduled per lane: each lane walks
 *                   its own member's blocks and takes the pair's next member when
 *                   its member is finished; block switches and refills run in a
 *                   shared service step (ndf_ksg_set_schedule).
 *                   Algorithm 1 only, like NDF_KSG_BLOCK;
 *   NDF_KSG_BRUTE   every member against every member of each pair.
 * count_evals != 0 makes the kernels count distance evaluations (read with
 * ndf_ksg_take_eval_count); it costs one atomic per warp per launch. */
typedef enum {
    NDF_KSG_BRUTE = 0,
    NDF_KSG_PRUNED = 1,
    NDF_KSG_BLOCK = 2,
    NDF_KSG_LANES = 3
} ndf_ksg_algorithm;
ndf_status ndf_set_ksg_algorithm(ndf_ctx* ctx, int algorithm, int count_evals);

/* NDF_KSG_LANES schedule: a warp checks every `every` scan steps (1..8,
 * default 5) whether to run its service step (block switches, refills), and
 * runs it when at least `switch_min` lanes wait (1..32, default 12) or none
 * scans.  Results do not depend on either.  NDF_ERR_ARG outside the ranges. */
ndf_status ndf_ksg_set_schedule(ndf_ctx* ctx, int switch_min, int every);

/* Distance evaluations counted since the last call (synchronizes; 0 when
 * counting is off). */
ndf_status ndf_ksg_take_eval_count(ndf_ctx* ctx, uint64_t* evals);

/* R KSG volumes in one persistent launch (the context's search): out[i*N + v] =
 * I(e^ref(ref_idx[i]); e^query(v)).  The exact searches take (reference,
 * vertex) pairs from one work counter; the brute-force search processes
 * references in groups that share each loaded query column and its sorted copy,
 * the group size and tile from ndf_ksg_autotune (defaults 4 references x 8
 * vertices).  ref_idx: R indices in host or device memory.  Host indices are
 * range-checked before anything is enqueued; device indices are checked by the
 * staging kernel (an index outside [0, N) leaves that reference's volume
 * meaningless and makes the next host check return NDF_ERR_ARG).  With device
 * indices and a device output the call enqueues only kernels and a memset --
 * no host copy, synchronisation or allocation once an earlier call with the
 * same R and fields has sized the scratch -- so it can be captured in a CUDA
 * graph on the context's stream and replayed. */
ndf_status ndf_mi_ksg_batch(ndf_ctx* ctx, int ref_field, int query_field, const int64_t* ref_idx,
                            int R, int k, float* out);

/* Times a few (references per CTA, vertices per tile) shapes of the batched
 * brute-force KSG kernel on a sample (8 references x up to 16384 query vertices) and keeps the
 * fastest for later ndf_mi_ksg_batch / ndf_train calls on this context.  The
 * chosen shape is written to *best_group / *best_tile (either may be NULL). */
ndf_status ndf_ksg_autotune(ndf_ctx* ctx, int ref_field, int query_field, int k, int* best_group,
                            int* best_tile);

/* Autotuner of the exact search itself (row a7's "autotuned tiles" for the
 * exact searches): times NDF_KSG_BLOCK and NDF_KSG_LANES under a grid of
 * (switch_min, every) schedules on a sample of the given fields (8 references,
 * 24,576 query vertices; about 0.3 s at M = 1000) and sets the fastest as the
 * context's search and schedule.  Outputs may be NULL.  Results of every search
 * are identical, so only speed depends on the choice.  Errors as ndf_mi_ksg, and
 * NDF_ERR_OOM / NDF_ERR_CUDA for its scratch or launches. */
ndf_status ndf_ksg_autotune_search(ndf_ctx* ctx, int ref_field, int query_field, int k,
                                   int* algorithm, int* switch_min, int* every);

/* Test hook for one (reference, query) pair of the KSG path above: writes, in
 * member order, eps[M] (k-th-neighbour distance), nx[M], ny[M] (marginal
 * counts) and *mi (the FP64 estimate before rounding to FP32).  All four
 * outputs are host pointers (any may be NULL).  Runs the same kernel as
 * ndf_mi_ksg on a one-vertex range and synchronizes. */
ndf_status ndf_ksg_debug_pair(ndf_ctx* ctx, int ref_field, int query_field, int64_t ref_idx,
                              int64_t query_idx, int k, float* eps, int32_t* nx, int32_t* ny,
                              double* mi);

/* The same hook for algorithm 2: ex[M], ey[M] (marginal extents of each
 * member's neighbour set), nx[M], ny[M] (non-strict counts) and *mi. */
ndf_status ndf_ksg2_debug_pair(ndf_ctx* ctx, int ref_field, int query_field, int64_t ref_idx,
                               int64_t query_idx, int k, float* ex, float* ey, int32_t* nx,
                               int32_t* ny, double* mi);

/* ---- grids split across GPUs (z-slabs) ------------------------------------ */

/* Given the reference vertex's member column, every vertex is an independent
 * problem (Sec. 3: R(p_ref, .) vertex by vertex), so a grid split into z-slabs
 * over several GPUs exchanges one M-float column per reference: the GPU whose
 * slab holds the reference vertex reads it with ndf_field_column and sends it;
 * every GPU computes its own slab with ndf_pearson_column / ndf_mi_ksg_column.
 * The column is staged as a one-vertex field whose statistics come from the
 * same per-vertex kernel as a loaded field's, so a slab's volume is bit-equal
 * to the same vertex range of ndf_pearson / ndf_mi_ksg on the whole grid. */

/* The M member values of one vertex of a loaded field: out[m] = e_m(vertex).
 * out: M floats, host or device.  NDF_ERR_ARG for an unknown field or a vertex
 * outside [0, N); NDF_ERR_STATE for a freed field. */
ndf_status ndf_field_column(ndf_ctx* ctx, int field_id, int64_t vertex, float* out);

/* ndf_pearson with the reference given as its member column (M floats of the
 * query field's member count, host or device, finite) instead of a vertex:
 * out[v] = r(ref_column, e^query(v)) for the N vertices of the query field.
 * Errors as ndf_pearson, and NDF_ERR_ARG for a null column. */
ndf_status ndf_pearson_column(ndf_ctx* ctx, const float* ref_column, int query_field, float* out);

/* ndf_mi_ksg (algorithm 1, the context's search) with the reference given as
 * its member column, as ndf_pearson_column.  Errors as ndf_mi_ksg. */
ndf_status ndf_mi_ksg_column(ndf_ctx* ctx, const float* ref_column, int query_field, int k,
                             float* out);

/* ---- neural dependence field (Sec. 4) ------------------------------------ */

/* Errors of the model calls in this section and the next: NDF_ERR_ARG for a
 * null model or pointer, B < 1 or R < 1, a reference index outside [0, N), an
 * unknown measure, decode mode or merge, grid dimensions or a training
 * configuration out of range, or k / M outside the KSG limits for MI targets;
 * NDF_ERR_STATE for a freed field; NDF_ERR_OOM / NDF_ERR_CUDA for failed
 * allocations, cuBLAS set-up, launches or copies; NDF_ERR_IO for model files
 * that cannot be opened, written, or are not (complete) model files of the
 * same parameter count. */

typedef struct ndf_model ndf_model; /* opaque; owned by the caller, freed by ndf_model_free */

/* Dependence measure a network learns. */
typedef enum { NDF_MEASURE_PEARSON = 0, NDF_MEASURE_MI_KSG = 1 } ndf_measure;

/* Training configuration (Sec. 4.3); ndf_train_cfg_default fills the values in
 * brackets.  The network is fixed at 4 dense feature-grid levels x 16 BF16
 * features (res[] points per axis, corner-aligned on [-1,1]^3), the merged
 * input [f_ref*f_q ; f_ref+f_q] (128), 3 hidden ReLU layers of 128 and one
 * output (tanh for Pearson, softplus for MI). */
typedef struct {
    int res[4];               /* grid points per axis per level [32, 64, 128, 256] */
    int64_t n_triples;        /* (reference, query, target) training triples [2^26] */
    int64_t batch;            /* pairs per Adam step [2^18] */
    int64_t refs_per_group;   /* references per generation group [128] */
    int64_t queries_per_group;/* query vertices per group [8192] */
    int max_passes;           /* passes over the triples [50] */
    int patience;             /* passes without improvement before lr x 0.1 [5] */
    int max_decays;           /* stop after this many decays [2] */
    float lr, beta1, beta2, eps; /* Adam [3e-4, 0.9, 0.999, 1e-8] */
    uint64_t seed;            /* triples, pass orders, initial weights [20230705] */
    double time_budget_s;     /* stop training after this many seconds (0: none) [0] */
    int32_t continuous;       /* 0: grid-vertex pairs, generated once; 1: uniform random
                                 positions with trilinear samples (ndf_sample_triples),
                                 n_triples fresh pairs every pass (Sec. 4.3) [0] */
    int32_t hash_tf32;        /* kept for layout compatibility and ignored: ndf_hash_train's
                                 dense layers are the library's own FP32 products [1] */
} ndf_train_cfg;

/* What a model is and how it was trained. */
typedef struct {
    int measure;
    int res[4];
    int64_t X, Y, Z;          /* ensemble grid the model decodes */
    int64_t param_count, grid_params;
    int64_t network_bytes;    /* decoding footprint: BF16 grid and weights, FP32 rest */
    int64_t training_bytes;   /* FP32 master + gradient + Adam moments + BF16 grid */
    int64_t adam_steps;
    int passes;
    double last_loss;         /* mean L1 loss of the last pass */
    int64_t n_triples;
    double gen_seconds, train_seconds;
} ndf_model_info_t;

void ndf_train_cfg_default(ndf_train_cfg* cfg);

/* Training samples at continuous positions (Sec. 4.3): n independent pairs of
 * uniform random positions p_ref, p_q in [-1,1]^3 (a 2^-23 grid; seeded), the
 * member columns of ref_field at p_ref and of query_field at p_q by trilinear
 * interpolation (vertex i of an axis of n at -1 + 2 i / (n - 1); FP32 in a fixed
 * order: u = ((p + 1) * 0.5) * (n - 1) clamped, i0 = min(floor(u), n - 2),
 * w = u - i0, a * (1 - w) + b * w along x, y, z), and the target R(p_ref, p_q):
 * Pearson r (Eq. 1, FP64 sums) or KSG MI (algorithm 1, k; the pruned search).
 * Writes pref[n][3], pq[n][3], target[n] (host or device; host outputs
 * synchronize).  Errors: NDF_ERR_ARG for bad ids, measure, k or n. */
ndf_status ndf_sample_triples(ndf_ctx* ctx, int ref_field, int query_field, int measure, int k,
                              int64_t n, uint64_t seed, float* pref, float* pq, float* target);

/* Learn Phi(p_ref, p_q) ~ R(p_ref, p_q) (Eq. 3, L1 loss, Adam) for the
 * reference field / query field pair (the self-correlation field when they
 * are the same, Sec. 3; a cross-variable field otherwise, Sec. 6.4).  Targets
 * come from this library's exact estimators (Pearson, or KSG MI with k) on
 * seeded uniform vertex pairs; positions are vertex-aligned in [-1,1]^3.
 * cfg may be NULL (defaults).  The new model is returned in *out. */
ndf_status ndf_train(ndf_ctx* ctx, int ref_field, int query_field, int measure, int k,
                     const ndf_train_cfg* cfg, ndf_model** out);

/* Decode a full dependence volume for one reference vertex (Sec. 5):
 * out[v] = Phi(p(ref_idx), p(v)) for all N vertices of the model's grid.
 * out: N floats, host or device. */
ndf_status ndf_infer(ndf_model* model, int64_t ref_idx, float* out);

/* R volumes in one launch: out[i*N + v] for R host reference indices. */
ndf_status ndf_infer_batch(ndf_model* model, const int64_t* ref_idx, int R, float* out);

/* Save / load a model (FP32 parameters and Adam state, versioned binary). */
ndf_status ndf_model_save(ndf_model* model, const char* path);
ndf_status ndf_model_load(ndf_ctx* ctx, const char* path, ndf_model** out);
void ndf_model_free(ndf_model* model);
ndf_status ndf_model_info(const ndf_model* model, ndf_model_info_t* info);

/* Lower-level calls (used by the tests and the benchmark).  A fresh model
 * over an X x Y x Z grid: grid features U(-1e-4, 1e-4), weights He-uniform,
 * biases 0, from a counter-based generator keyed by seed. */
ndf_status ndf_model_create(ndf_ctx* ctx, const int res[4], int measure, uint64_t seed, int64_t X,
                            int64_t Y, int64_t Z, ndf_model** out);
/* Number of FP32 parameters; layout: grid levels (point-major, 16 features),
 * W1 [128][128] ([out][in]), b1, W2, b2, W3, b3, w4 [128], b4. */
int64_t ndf_model_param_count(const ndf_model* model);
ndf_status ndf_model_get_params(ndf_model* model, float* out);      /* host or device */
ndf_status ndf_model_set_params(ndf_model* model, const float* in); /* host or device */
/* One step on B explicit position pairs (p_ref, p_query: [B][3] in [-1,1]^3)
 * with targets: writes the mean L1 loss and (if grad_out) dL/dparams in the
 * parameter layout; with update != 0 also applies one Adam step at rate lr. */
ndf_status ndf_model_step(ndf_model* model, const float* p_ref, const float* p_query,
                          const float* target, int64_t B, float lr, int update, double* loss_out,
                          float* grad_out);
/* Phi for B explicit position pairs; out: B floats, host or device. */
ndf_status ndf_model_forward(ndf_model* model, const float* p_ref, const float* p_query,
                             int64_t B, float* out);

/* ---- the paper's NDF architecture (Sec. 4.1-4.2, Fig. 2; row f2) ---------- */

/* Hidden-layer activations: ReLU, Snake x + sin^2 x, SnakeAlt x / 2 + sin^2 x. */
typedef enum { NDF_ACT_RELU = 0, NDF_ACT_SNAKE = 1, NDF_ACT_SNAKEALT = 2 } ndf_activation;

/* Feature merge (Sec. 4.1): the paper's element-wise product, and the
 * alternatives it compares against (sum, absolute difference, concatenation). */
typedef enum {
    NDF_MERGE_PRODUCT = 0,
    NDF_MERGE_SUM = 1,
    NDF_MERGE_ABSDIFF = 2,
    NDF_MERGE_CONCAT = 3
} ndf_merge;

/* Input embedding [p, Fourier features (Eq. 4: sin / cos(2^i pi p_j), i < n_freq),
 * hash-grid features] -> encoder MLP (enc_layers linear layers of `width`,
 * activation between them) -> element-wise product of the two positions'
 * latents -> decoder MLP (dec_layers, last to 1) -> tanh (Pearson) or softplus
 * (MI).  Hash grid: `levels` levels of base_res * 2^l points per axis
 * (corner-aligned on [-1,1]^3), min(2^log2_table, R^3) entries of `feat`
 * features each (dense index when the level fits, else the spatial hash
 * x*1 ^ y*2654435761 ^ z*805459861 mod 2^T).  ndf_hash_arch_default gives the
 * paper's 6 levels from 16^3, L = 12, 6 + 6 layers of 128, SnakeAlt, product
 * merge; the table size defaults to 2^22 per level (the paper's 2^30 would
 * need 51 GB of FP32 training state).  enc_layers = 0 is the grid-only ablation
 * (Sec. 6.4: the latent is the embedding itself). */
typedef struct {
    int32_t levels, base_res, log2_table, feat, n_freq, width, enc_layers, dec_layers, act;
    int32_t merge; /* ndf_merge */
} ndf_hash_arch;
void ndf_hash_arch_default(ndf_hash_arch* arch);

typedef struct ndf_hash_model ndf_hash_model;

/* A model decoding grids of X x Y x Z vertices.  cross = 0: one encoder and
 * grid for both positions (self fields, Phi(p1, p2) = Phi(p2, p1) exactly);
 * cross = 1: separate encoders (0 reference, 1 query).  Parameters follow the
 * layout of the oracle (per encoder: level tables, then W[out][in], b per layer;
 * then the decoder layers), FP32, with Adam moments.  Initialisation: tables
 * U(-0.1, 0.1), weights U(+-sqrt(6 / fan_in)) except the first encoder layer's
 * weights on the Fourier columns, which start at 0.1 of that scale, biases 0,
 * the last decoder layer 0 (seeded). */
ndf_status ndf_hash_model_create(ndf_ctx* ctx, const ndf_hash_arch* arch, int measure, int cross,
                                 uint64_t seed, int64_t X, int64_t Y, int64_t Z,
                                 ndf_hash_model** out);
void ndf_hash_model_free(ndf_hash_model* m);
int64_t ndf_hash_model_param_count(const ndf_hash_model* m);
ndf_status ndf_hash_model_get_params(ndf_hash_model* m, float* out);      /* host or device */
ndf_status ndf_hash_model_set_params(ndf_hash_model* m, const float* in); /* host or device */

/* out[B] = network(pr[b], pq[b]); pr, pq [B][3] positions in [-1,1]^3. */
ndf_status ndf_hash_model_forward(ndf_hash_model* m, const float* pr, const float* pq, int64_t B,
                                  float* out);

/* One step of the mean L1 loss (Eq. 3): gradient of every parameter (copied to
 * grad_out when not NULL), the loss in *loss_out, and with apply != 0 an Adam
 * update (beta 0.9 / 0.999, eps 1e-8) with learning rate lr. */
ndf_status ndf_hash_model_step(ndf_hash_model* m, const float* pr, const float* pq,
                               const float* target, int64_t B, float lr, int apply,
                               float* grad_out, double* loss_out);

/* Training on continuous-position samples (ndf_sample_triples), n_triples fresh
 * pairs every pass, Adam and the plateau schedule of cfg (Sec. 4.3). */
ndf_status ndf_hash_train(ndf_ctx* ctx, int ref_field, int query_field, int measure, int k,
                          const ndf_hash_arch* arch, const ndf_train_cfg* cfg,
                          ndf_hash_model** out);

/* Passes, last pass loss, sampling and training seconds, Adam steps. */
ndf_status ndf_hash_model_info(const ndf_hash_model* m, int* passes, double* last_loss,
                               double* gen_seconds, double* train_seconds, int64_t* adam_steps);

/* The dependence volume of one reference vertex (vertex-aligned positions,
 * Sec. 5): out[N] (host or device), N = X * Y * Z.  The reference latent is
 * encoded once; the path is the one ndf_hash_set_decode selected. */
ndf_status ndf_hash_infer(ndf_hash_model* m, int64_t ref_idx, float* out);

/* R volumes, out[R][N] (host or device); ref_idx: R host indices in [0, N).
 * The tensor-core path decodes up to 64 references per launch (one CTA row per
 * reference).  NDF_ERR_ARG for an index out of range. */
ndf_status ndf_hash_infer_batch(ndf_hash_model* m, const int64_t* ref_idx, int32_t R, float* out);

/* Decoding path of ndf_hash_infer / ndf_hash_infer_batch.
 *   NDF_HASH_DECODE_FP32: FP32 layers (cuBLAS SGEMM), the same arithmetic as
 *     ndf_hash_model_forward; queries in chunks of 65536.
 *   NDF_HASH_DECODE_TC: one persistent tcgen05 kernel per launch runs the whole
 *     chain for 128-vertex tiles (BF16 operands, FP32 accumulation in TMEM;
 *     embedding, biases, activations, merge and output layer in FP32).  Needs
 *     width 128, at most 128 embedding inputs and a product / sum / |difference|
 *     merge (NDF_ERR_ARG otherwise).
 *   cache_queries != 0 (TC only; at least one encoder and two decoder layers):
 *     the N query latents are encoded once per parameter change and kept on
 *     the device (N x 128 FP32); each reference then runs only the merge and the
 *     decoder.  The results equal the uncached TC path's.
 * A new model starts in NDF_HASH_DECODE_TC when its architecture allows it,
 * else in FP32, without the cache. */
typedef enum { NDF_HASH_DECODE_FP32 = 0, NDF_HASH_DECODE_TC = 1 } ndf_hash_decode;
ndf_status ndf_hash_set_decode(ndf_hash_model* m, int32_t mode, int32_t cache_queries);
int32_t ndf_hash_get_decode(const ndf_hash_model* m); /* the mode, -1 for NULL */

/* ---- headless volume rendering (Sec. 5, Sec. 6.5) -------------------------- */

/* Errors: NDF_ERR_ARG for a null volume, configuration or image, a volume with
 * an axis of fewer than 2 vertices or more than 2^31 vertices in all, a bad
 * image size or render
 * configuration, an eye at the target, or an up vector parallel to the view
 * direction; NDF_ERR_OOM / NDF_ERR_CUDA as above. */

/* Direct volume rendering with a transfer function, or an iso-surface. */
typedef enum { NDF_RENDER_DVR = 0, NDF_RENDER_ISO = 1 } ndf_render_mode;

typedef struct {
    float eye[3], target[3], up[3]; /* pinhole camera in the volume's [-1,1]^3 frame */
    float fov_y_deg;                /* vertical field of view, (0, 180) degrees */
    int32_t width, height;          /* image size in pixels */
    float step;                     /* ray-march step, > 0 (box units) */
    int32_t mode;                   /* ndf_render_mode */
    float iso;                      /* iso value (NDF_RENDER_ISO) */
    float vmin, vmax;               /* transfer-function domain, vmax > vmin */
    float background[4];            /* RGBA behind the volume */
    float ambient;                  /* iso-surface ambient term in [0, 1] */
    int32_t n_tf;                   /* transfer-function entries, >= 1 */
    const float* tf;                /* host [n_tf][4] RGBA; A = opacity per unit length */
} ndf_render_cfg;

/* Ray-marches the dependence volume vol_a[Z][Y][X] (host or device; vertex i of
 * an axis of n vertices sits at -1 + 2 i / (n - 1), as ndf_infer decodes), or
 * the difference vol_a - vol_b of two reference fields when vol_b is not NULL
 * (Sec. 6.5), into out_rgba[height][width][4] (FP32, host or device).
 * Samples: trilinear, at t0 + (k + 1/2) step along each ray inside [-1,1]^3.
 * DVR: alpha = 1 - exp(-A step), front-to-back compositing over the background.
 * ISO: first sign change of (value - iso), linear refinement, central-difference
 * normal (h = step) turned to the viewer, colour tf(iso) * (ambient +
 * (1 - ambient) max(0, n . -dir)).  Requires X, Y, Z >= 2 (NDF_ERR_ARG
 * otherwise, and for a bad configuration).  Host volumes are copied to context
 * scratch; synchronous only when out_rgba is a host pointer. */
ndf_status ndf_render_volume(ndf_ctx* ctx, const float* vol_a, const float* vol_b, int64_t X,
                             int64_t Y, int64_t Z, const ndf_render_cfg* cfg, float* out_rgba);

/* ---- allocation-free variant --------------------------------------------- */

/* Largest member count ndf_pearson_noalloc accepts. */
#define NDF_NOALLOC_MAX_M 16384

/* Pearson volume that allocates no memory at all (no cudaMalloc, no cudaFree,
 * no allocating library call), for callers that cannot allocate device memory:
 * applications whose own allocator or pool owns the device budget, or whose
 * frame loop cannot absorb the device-wide synchronisation an allocation may
 * cause.  The paper has no counterpart; it is an addition of this library.
 *
 * Same result as ndf_pearson (Eq. 1 for every vertex, FP32, clamped, 0 for
 * zero variance) but without a context or a loaded ensemble: ref_field and
 * query_field are caller-owned DEVICE buffers float[M][N] (member-major, may be
 * the same buffer), out is a caller-owned DEVICE buffer of N floats, and the
 * work is enqueued on cuda_stream (NULL = legacy default stream); the call
 * returns without synchronising.  The query statistics are formed in the same
 * pass, so nothing needs to be loaded first.
 *
 * Scratch: a fixed 64 KB file-scope device array (NDF_NOALLOC_MAX_M floats and
 * two doubles) that every GPU loading the library holds until the process
 * exits.  Each call outside stream capture looks up that array's device
 * address on the current device (cudaGetSymbolAddress); a call during capture
 * uses the address found by the last call outside capture, so make the first
 * call on a device, and the first call after a device reset, before any stream
 * capture (otherwise NDF_ERR_STATE).  All calls share the array and each
 * rewrites what it reads, so calls that overlap on the GPU (other streams,
 * other threads) race: serialise them.
 *
 * All three buffers must be memory of the CURRENT device (or managed memory):
 * a buffer of another GPU is rejected, since the kernels read without peer
 * access.
 *
 * Errors: NDF_ERR_ARG for a null pointer, a pointer that is not device memory
 * of the current device, M < 2, M > NDF_NOALLOC_MAX_M, N < 1 or ref_idx
 * outside [0, N); NDF_ERR_STATE for the first call on a device made during
 * stream capture; NDF_ERR_CUDA when the set-up or a launch fails, and also,
 * without launching anything, when a CUDA error from the caller's earlier work
 * is already pending on this thread (it is left pending for the caller to
 * read).  There is no context, so no error string. */
ndf_status ndf_pearson_noalloc(const float* ref_field, const float* query_field, int64_t M,
                               int64_t N, int64_t ref_idx, float* out, void* cuda_stream);

/* The pointer rule of ndf_pearson_noalloc as a pure host function (a test
 * hook; no CUDA call): 1 when a buffer with these attributes is accepted --
 * managed memory, or device memory whose device equals the current device --
 * else 0.  The paper has no counterpart. */
int ndf_noalloc_pointer_usable(int is_device, int is_managed, int ptr_device, int current_device);

#ifdef __cplusplus
}
#endif
#endif /* NDF_H */
