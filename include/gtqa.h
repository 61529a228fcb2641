/*
 * gtqa.h -- C ABI of the GB300 graph tensor-network quantum annealer (GTQA) hot path.
 *
 * Method: arXiv:2409.12240, "Large-scale quantum annealing simulation with tensor
 * networks and belief propagation".  One annealing layer is
 *   (1) the Trotterised interaction layer U_Z: one two-qubit gate per edge, applied
 *       by the simple update with truncation back to bond dimension chi
 *       (App. E, App. D Algorithm "Truncation", App. F Eq. (discretizatoion));
 *   (2) the mixing layer U_X: one single-qubit gate per vertex (Sec. II D);
 *   (3) belief propagation on the symmetric-gauge network from warm-start
 *       messages (Sec. II C Eq. (symmetric_gauge), Eq. (reconstructed_messages);
 *       App. B Algorithm "Belief propagation", flooding schedule);
 *   (4) Vidal gauge finding from the messages (App. D Algorithm "Vidal gauge finding");
 * plus single-qubit reduced density matrices and the sign read-out
 * (Eq. (partial_dens), Eq. (bp_approx), Eq. (rounding_rule)).
 *
 * Conventions shared by every call:
 *  - Vertices 0..n-1, edges 0..m-1 given as pairs (u, v); u is the edge's "first"
 *    endpoint.  Degree <= 3.  A vertex's bond slots are its incident edges in
 *    ascending edge id; missing slots (degree < 3) are phantom bonds of dimension 1.
 *  - Bond storage is padded to CHI = smallest of {2, 4, 8} >= chi; entries beyond a
 *    bond's current dimension are exactly zero.
 *  - Device work runs in three persistent kernels (gates, BP, regauge), each launched
 *    cooperatively with one block per SM; their grid barriers poll with a bound and
 *    report GTQA_ERR_TIMEOUT instead of hanging.
 *  - Gamma layout: complex128 interleaved (re, im) array [n][2][CHI][CHI][CHI],
 *    index (i, j_slot0, j_slot1, j_slot2); lambda: float64 [m][CHI], descending;
 *    messages: complex128 [2m][CHI][CHI], row 2e holds m_{u->v}, row 2e+1 holds
 *    m_{v->u} for edge e = (u, v); m[j][j'] pairs j with the ket, j' with the bra.
 *  - Physical index i = 0 is |0> (Z = +1, x = +1), i = 1 is |1> (Sec. III A).
 *  - Pointers named *_out or taking arrays may be host or device memory; the library
 *    detects which with cudaPointerGetAttributes.  The caller owns every array it
 *    passes; inputs are copied before the call returns.
 *  - All device work is ordered on the stream given in gtqa_options.cuda_stream.
 *    Calls that return values to the host synchronise that stream.
 *  - Every call returns GTQA_OK (0) or an error code.  Errors other than
 *    GTQA_ERR_INVALID_ARG and GTQA_ERR_NOT_CONVERGED are sticky: the state refuses
 *    further work until gtqa_destroy.  A state is not thread-safe.
 */
#ifndef GTQA_H
#define GTQA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GTQA_OK 0
#define GTQA_ERR_INVALID_ARG 1   /* bad size, index, degree > 4, duplicate edge, bad colouring, NaN input */
#define GTQA_ERR_NOT_CONVERGED 2 /* BP hit max_iter before dist/|E| < tol; state and outputs valid */
#define GTQA_ERR_NUMERIC 3       /* NaN or Inf detected on the device */
#define GTQA_ERR_OOM 4           /* device allocation failed */
#define GTQA_ERR_CUDA 5          /* a CUDA runtime call failed */
#define GTQA_ERR_TIMEOUT 6       /* a bounded device-side wait gave up */
#define GTQA_ERR_UNSUPPORTED 7   /* chi or precision not built into this library */

/* arithmetic modes */
#define GTQA_FP64 0   /* complex128 everywhere */
#define GTQA_MIXED 1  /* complex64 tensors and BP contractions; FP64 QR/SVD, gauge roots, normalisation.
                         Messages are held as m0 + delta: m0 = diag(lambda)/sum(lambda) (exact),
                         delta in complex64; get/set_state convert to and from complex128. */
#define GTQA_C64 2    /* complex64 with every step in FP32, including the QR/SVD, gauge roots and
                       * normalisation (a reference point for the precision split; plain kernels,
                       * one instance, degree 3 with chi <= 16 or degree 4 with chi <= 4; default
                       * cut-offs 1e-7 on singular values and 1e-6 on message eigenvalues) */

/* flags of gtqa_bp_sweep */
#define GTQA_BP_WARM_START 1u  /* start from m_{a->b} = diag(lambda_ab)/sum(lambda_ab) (Eq. reconstructed_messages) */
#define GTQA_BP_REGAUGE 2u     /* afterwards run Vidal gauge finding (App. D) */
#define GTQA_BP_DEFAULT 3u

typedef struct gtqa_state gtqa_state;

typedef struct gtqa_options {
    int32_t precision;   /* GTQA_FP64, GTQA_MIXED or GTQA_C64 */
    int32_t reserved0;   /* must be 0 */
    double svd_cutoff;   /* singular values <= svd_cutoff * s_0 are dropped; <= 0 selects the
                            precision's default: 1e-14, or 1e-7 for GTQA_C64 */
    double eig_cutoff;   /* message eigenvalues <= eig_cutoff * w_max count as zero; <= 0 selects
                            1e-13, or 1e-6 for GTQA_C64 */
    void* cuda_stream;   /* cudaStream_t for all work; NULL selects the legacy default stream */
} gtqa_options;

typedef struct gtqa_stats_t {
    int64_t layers;          /* gtqa_trotter_layer calls completed */
    int64_t gates;           /* two-qubit gates applied (all instances) */
    int32_t last_bp_iters;   /* sweeps run by the last gtqa_bp_sweep (max over instances) */
    int32_t not_converged;   /* instances that reached max_iter in the last gtqa_bp_sweep */
    double last_bp_dist;     /* dist/|E| after the last sweep (max over instances), App. B */
    double discarded_weight; /* sum over gates of sum_{dropped} s^2 / sum s^2 */
    double log_fidelity;     /* sum over gates of log f, f = (1 - discarded)^2, Eq. (gate_fidelity) */
    int64_t svd_pairs;       /* column pairs examined by the gate-core FP64 Jacobi sweeps (the polish
                                in GTQA_MIXED; work counter) */
    int64_t svd_rotations;   /* rotations applied by the gate-core Jacobi SVDs (work counter) */
    int64_t bp_sweeps;       /* BP sweeps run since creation (sum over calls, max over instances) */
    int64_t launches;        /* kernels launched by the library since creation */
    int64_t bp_calls;        /* BP runs since creation (one per layer in gtqa_anneal) */
    int64_t bp_not_converged_calls; /* BP runs in which some instance reached max_iter */
    int64_t bp_exact_passes; /* separate passes computing the exact trace-norm distance of a sweep
                                (persistent path: when a sweep's lower bound falls under tol) */
    int64_t regauge_svd_sweeps; /* Jacobi sweeps of the regauge's eigen-decompositions and SVDs
                                   (persistent path; work counter) */
    int32_t gate_svd_sweeps_max;      /* most FP64 Jacobi sweeps of one gate-core SVD since creation
                                         (the FP64 polish sweeps in GTQA_MIXED, whose sweeps after
                                         the first run only the schedule steps that still rotate
                                         by more than the stop threshold; persistent path) */
    int32_t gate_svd_sweeps32_max;    /* GTQA_MIXED: most FP32 preconditioning sweeps of one gate-core SVD */
    int32_t regauge_svd_sweeps_max;   /* the same two maxima for the regauge's decompositions */
    int32_t regauge_svd_sweeps32_max;
} gtqa_stats_t;

/* kernels timed by the optional profiler (gtqa_profile) */
#define GTQA_K_TROTTER 0    /* gates_kernel: the gate phases of one layer (gtqa_trotter_layer, gtqa_anneal) */
#define GTQA_K_BP 1         /* bp_kernel: warm start and BP sweeps of one BP run */
#define GTQA_K_REGAUGE 2    /* regauge_kernel: Vidal gauge finding */
#define GTQA_K_MARGINALS 3  /* marginals_kernel */
#define GTQA_K_COUNT 4

/* Fill *opt with defaults: FP64, default cut-offs, default stream. */
void gtqa_options_init(gtqa_options* opt);

/*
 * Create the state |+>^N (all bond dimensions 1, Sec. III A) of one problem instance.
 *   n, m       vertices and edges
 *   edges      host int32 [m][2]; 0 <= u, v < n, u != v, no repeated pair, degree <= 4
 *   colour     host int32 [m] proper edge colouring (each colour a matching), or NULL
 *              for the library's own (gtqa_edge_colouring).
 *              Gates run colour by colour, ascending (the paper leaves the order open).
 *   J, h       host float64 couplings [m] and fields [n] of Eq. (objective_function)
 *   chi        maximal bond dimension, 1 <= chi <= 16 (storage 2, 4, 8 or 16)
 *   opt        options or NULL for defaults
 *   out        receives the new state; *out is NULL on failure
 * Graphs with a vertex of degree 4 (the random 4-regular graphs of Sec. V) get vertex tensors
 * with four bonds, Gamma [n][2][CHI]^4; 8 < chi <= 16 gets storage bond dimension 16.  These
 * states, and every state in the GTQA_C64 precision, run on plain per-phase kernels and hold
 * one instance.  The shapes built there are: FP64 and GTQA_MIXED with degree 4 and chi <= 4, or
 * degree 3 and 8 < chi <= 16; GTQA_C64 with degree 3 and chi <= 16, or degree 4 and chi <= 4.
 * Anything else
 * returns GTQA_ERR_UNSUPPORTED.  On a plain-path state gtqa_autotune and gtqa_anneal_graph
 * return GTQA_ERR_UNSUPPORTED (there is no persistent launch to tune or capture), and so does
 * gtqa_apply_gates at chi > 8; every other call works as documented.  Its BP reads the
 * distance on the host after every sweep, and gtqa_anneal_policy reads R on the host.
 */
int gtqa_create(int32_t n, int32_t m, const int32_t* edges, const int32_t* colour,
                const double* J, const double* h, int32_t chi,
                const gtqa_options* opt, gtqa_state** out);

/*
 * Create B independent instances that evolve together (one launch per phase covers
 * all of them).  Arrays are concatenations over instances: n[B], m[B]; edges (local
 * vertex ids per instance) sum(m) pairs; colour sum(m) or NULL; J sum(m); h sum(n).
 * BP convergence is tracked per instance: dist_b/|E_b| < tol.
 */
int gtqa_create_batch(int32_t B, const int32_t* n, const int32_t* m, const int32_t* edges,
                      const int32_t* colour, const double* J, const double* h, int32_t chi,
                      const gtqa_options* opt, gtqa_state** out);

/*
 * One Trotter layer U_X(t_X) U_Z(t_Z) with t_Z = dt * tau and t_X = dt * (1 - tau)
 * (App. F Eq. (discretizatoion); tau = k/K is the Ising weight of layer k).
 * Each edge gate exp(-i t_Z (J Z_a Z_b + h_a/D_a Z_a + h_b/D_b Z_b)) is applied by the
 * simple update (App. E) and truncated to chi (App. D "Truncation"); then
 * exp(-i t_X X) acts on every vertex (Sec. II D).  Asynchronous.
 */
int gtqa_trotter_layer(gtqa_state* s, double tau, double dt);

/*
 * Belief propagation on T_a = Gamma_a prod lambda^{1/2} (Eq. (symmetric_gauge)),
 * flooding schedule, Eq. (local_consistency) with unit-trace normalisation, until
 * dist/|E| < tol or max_iter sweeps (App. B).  flags: GTQA_BP_WARM_START starts from
 * the reconstructed messages, otherwise from the state's current messages;
 * GTQA_BP_REGAUGE then applies Vidal gauge finding (App. D), which rewrites Gamma
 * and lambda.  iters_out / dist_out (nullable host pointers) receive the sweeps run
 * and the final dist/|E| (max over instances).  Synchronises the stream.
 * Returns GTQA_ERR_NOT_CONVERGED if some instance reached max_iter.
 */
int gtqa_bp_sweep(gtqa_state* s, double tol, int32_t max_iter, uint32_t flags,
                  int32_t* iters_out, double* dist_out);

/* Vidal gauge finding (App. D) from the state's current messages.  Asynchronous. */
int gtqa_regauge(gtqa_state* s);

/*
 * Layers k_begin..k_end (1-based, k_end <= K) of the K-layer linear anneal with step dt:
 * for each k, gtqa_trotter_layer(tau = k/K, dt) followed by gtqa_bp_sweep(tol, max_iter,
 * GTQA_BP_DEFAULT): three cooperative launches per layer and no host synchronisation
 * (BP stops on the device).  Asynchronous: BP counters go to gtqa_stats (bp_calls,
 * bp_not_converged_calls, bp_sweeps).
 */
int gtqa_anneal(gtqa_state* s, int32_t k_begin, int32_t k_end, int32_t K, double dt, double tol,
                int32_t max_iter);

/*
 * Autotuner of the launch shapes.  Each of the three phase kernels (gates, BP, regauge) is a
 * persistent cooperative launch of `grid` blocks, one per SM at most, in one of a few compiled
 * launch-shape variants (threads per block and team sizes; see gtqa_launch_shape).  For each
 * kernel in turn, gtqa_autotune times one launch of the layer (tau, dt) with BP to
 * (tol, max_iter) from the state's current contents, for every variant whose shared memory fits
 * on an SM and, per variant, each candidate grid: all SMs and, when the kernel's work fits in one
 * round of that variant's teams, 7/8 ... 1/2 of them and the fewest blocks that cover it.  The
 * earlier phases of the layer run untimed first, so that each kernel sees its real inputs.  The
 * median of three runs decides, and the fastest (variant, grid) pair is kept for the state.  The
 * state is snapshotted once (into device memory when a copy fits in free memory, else into host
 * memory), its contents and statistics are restored afterwards, and a layer graph captured by
 * gtqa_anneal_graph is dropped (the next call captures the new shapes).  grid_out (nullable,
 * 3 ints) receives the chosen grid sizes.  Results do not depend on the grid; across variants
 * they differ only in the rounding order of BP's contraction and distance sums.  Synchronises.
 * Returns GTQA_ERR_UNSUPPORTED for a plain-path state (gtqa_create).
 */
int gtqa_autotune(gtqa_state* s, double tau, double dt, double tol, int32_t max_iter, int32_t* grid_out);

/* Set the grid sizes (blocks of the gates, BP and regauge kernels, each 1..number of SMs), for
 * example to apply gtqa_autotune's choice from another state of the same shape.  Drops a
 * captured layer graph. */
int gtqa_set_grid(gtqa_state* s, const int32_t* grid);

/*
 * Launch-shape variants (3 ints: gates, BP, regauge).  The gates kernel has variants 0 and 1,
 * BP and regauge 0, 1 and 2; variant 0 is the default of gtqa_create_batch.  For CHI <= 4
 * (threads per block, BP vertex team, regauge-vertex team) are (512, 64, 32), (256, 64, 32) and
 * (512, 128, 64); for CHI = 8 they are (256, 256, 128), (512, 256, 128) and (512, 512, 256).
 * The gate-edge team (2 CHI^2 threads) and the regauge-edge team (CHI^2) are fixed.
 * GTQA_ERR_INVALID_ARG for an index out of range, GTQA_ERR_UNSUPPORTED when a variant's
 * shared memory does not fit on an SM (the state keeps its shapes) or for a plain-path state.
 * Drops a captured layer graph.
 */
int gtqa_set_shape(gtqa_state* s, const int32_t* variant);

/* The current launch table: out[4 k .. 4 k + 3] = grid blocks, shape variant, threads per
 * block and team size (gate edge, BP vertex, regauge vertex) of kernel k = gates, BP, regauge
 * (12 ints).  GTQA_ERR_UNSUPPORTED for a plain-path state. */
int gtqa_launch_shape(gtqa_state* s, int32_t* out);

/*
 * gtqa_anneal with the paper's occasional regauging (Sec. II C: the Vidal gauge is restored
 * when the local-orthogonality residual R of App. C grows too large).  After each layer's gates
 * R is evaluated on the device (as gtqa_residual, normalised by 2|E|; for a batch, over all
 * instances together).  BP from the warm start and Vidal gauge finding then run only if
 * R > r_threshold; otherwise they are skipped on the device, with no host synchronisation,
 * and the state keeps its simple-update gauge.  A negative threshold regauges every layer, as
 * gtqa_anneal does.  Skipped layers leave gtqa_stats' last-BP fields unchanged;
 * gtqa_regauge_counts reports how many layers were regauged and skipped.  Asynchronous.
 * On a plain-path state (gtqa_create) the host reads R after the gates of every layer and
 * launches BP and the regauge only when R > r_threshold; that loop synchronises once per layer
 * and returns GTQA_ERR_NUMERIC if R is NaN.
 * Returns GTQA_ERR_INVALID_ARG as gtqa_anneal or for a NaN threshold.
 */
int gtqa_anneal_policy(gtqa_state* s, int32_t k_begin, int32_t k_end, int32_t K, double dt, double tol,
                       int32_t max_iter, double r_threshold);

/* Layers regauged and skipped by gtqa_anneal_policy since creation.  Synchronises. */
int gtqa_regauge_counts(gtqa_state* s, int64_t* regauged, int64_t* skipped);

/*
 * gtqa_anneal replayed from a CUDA graph: the three launches of one layer (gates, BP,
 * regauge) are captured once (on a private stream) into a graph that the state keeps.  The
 * captured layer reads its index k from a device word, and its regauge launch stores k + 1,
 * so layers k_begin..k_end are one small kernel that sets k_begin followed by one graph launch
 * per layer on the state's stream.  The graph is kept for later calls with the same K, dt,
 * tol and max_iter (any layer range) and the same profiling setting; other values replace it.
 * The results are those of gtqa_anneal with the same arguments, bit for bit; the graph saves
 * the host-side launch cost and the device work is unchanged.  The graph carries events
 * between its three launches; with the profiler on (gtqa_profile) each replay is timed into
 * the gates, BP and regauge classes, its events being read before the next replay (a
 * multi-layer call then waits for each layer before launching the next) or by
 * gtqa_profile_read.  Otherwise asynchronous.  Returns GTQA_ERR_UNSUPPORTED if the launches could not be captured
 * (nothing is launched and the state stays usable) or for a degree-4 state, and
 * GTQA_ERR_INVALID_ARG as gtqa_anneal.
 */
int gtqa_anneal_graph(gtqa_state* s, int32_t k_begin, int32_t k_end, int32_t K, double dt, double tol,
                      int32_t max_iter);

/*
 * One Trotter layer in split form U_X(t_X_post) U_Z(t_Z) U_X(t_X_pre): the mixing gate
 * exp(-i t_X_pre X) on every vertex, then every edge gate of U_Z(t_Z) by the simple update
 * with truncation (App. E, App. D "Truncation"), then exp(-i t_X_post X) on every vertex
 * (Sec. II D).  gtqa_trotter_layer(tau, dt) is (0, dt tau, dt (1 - tau)).  The building
 * block of the product formulas beyond first order that Sec. V names.  Asynchronous.
 * Returns GTQA_ERR_INVALID_ARG for a non-finite angle.
 */
int gtqa_trotter_split(gtqa_state* s, double t_Z, double t_X_pre, double t_X_post);

#define GTQA_TROTTER_FIRST 1      /* U_X(t_X) U_Z(t_Z); reversed: U_Z(t_Z) U_X(t_X) */
#define GTQA_TROTTER_SYMMETRIC 2  /* U_X(t_X/2) U_Z(t_Z) U_X(t_X/2), second order */

/*
 * gtqa_anneal with a choice of product formula (Sec. V: higher-order and randomised
 * formulas).  Layer k (t_Z = dt k/K, t_X = dt (1 - k/K)) is gtqa_trotter_split with
 *   GTQA_TROTTER_FIRST:     (t_X_pre, t_X_post) = (0, t_X), or (t_X, 0) when reverse is
 *                           non-NULL and reverse[k - k_begin] != 0; drawing reverse[] as
 *                           fair coin flips gives the randomised first-order formula;
 *   GTQA_TROTTER_SYMMETRIC: (t_X/2, t_X/2); reverse must be NULL;
 * followed by BP from the warm start and the regauge, as in gtqa_anneal.  reverse is a
 * host array of k_end - k_begin + 1 bytes, read before the call returns.  Asynchronous.
 * Returns GTQA_ERR_INVALID_ARG for a bad range, order, or a reverse array with the
 * symmetric formula.
 */
int gtqa_anneal_ex(gtqa_state* s, int32_t k_begin, int32_t k_end, int32_t K, double dt, double tol,
                   int32_t max_iter, int32_t order, const uint8_t* reverse);

/*
 * Arbitrary two-qubit gates (Sec. II D, App. E): gate q acts on edge edge[q] = {u, v}, u and
 * v its endpoints in the order given at creation, with the 4x4 complex matrix
 * U[q][r][c] (r = 2 i_u + i_v, c = 2 i_u' + i_v'; host array of k x 16 complex128 as
 * interleaved re, im pairs, row-major).  Each gate is a simple update of the edge's bond
 * with truncation to chi (App. D "Truncation"); U need not be unitary.  Gates are applied in
 * list order: the host packs them into launches of gates with disjoint endpoints, a gate
 * going one launch after the latest earlier gate that shares a vertex with it, so the
 * result is that of the sequential list.  QR and SVD in FP64 in both precision modes.
 * Like gtqa_trotter_layer the call leaves the state out of the Vidal gauge: follow it with
 * gtqa_bp_sweep(..., GTQA_BP_DEFAULT) before reading marginals.  The discarded weight and
 * log-fidelity of each gate go to gtqa_stats.  Asynchronous; edge and U are read before
 * the call returns.  Returns GTQA_ERR_INVALID_ARG for k < 0, an edge outside [0, m) (global
 * ids in a batched state) or a non-finite entry.
 */
int gtqa_apply_gates(gtqa_state* s, int32_t k, const int32_t* edge, const double* U);

/*
 * Host-only: the launch layering gtqa_apply_gates uses for a gate list.  layer_out[q] is the
 * launch of gate q: one after the latest earlier gate sharing a vertex with it (0 if none).
 * Gates of one launch have disjoint endpoints, and gates sharing a vertex keep their order.
 * n_layers_out (nullable) receives the number of launches.  edges: host int32 [m][2]; edge:
 * host int32 [k], each in [0, m).
 */
int gtqa_gate_layers(int32_t n, int32_t m, const int32_t* edges, int32_t k, const int32_t* edge, int32_t* layer_out,
                     int32_t* n_layers_out);

/*
 * Arbitrary one-qubit gates (Sec. II D): Gamma_a[i] <- sum_i' W[q][i][i'] Gamma_a[i'] for
 * a = vertex[q], in list order (W: host array of k x 4 complex128, interleaved, row-major).
 * Gates on one vertex are composed on the host, then one launch applies every vertex's
 * product.  No truncation and no change of gauge class: the Vidal gauge is kept.
 * Asynchronous; returns GTQA_ERR_INVALID_ARG for k < 0, a vertex outside [0, n) or a
 * non-finite entry.
 */
int gtqa_apply_single_qubit_gates(gtqa_state* s, int32_t k, const int32_t* vertex, const double* W);

/*
 * BP-guided measurement sampling of a bitstring (Sec. IV A), for problems whose solutions
 * are degenerate so that the read-out of Eq. (rounding_rule) does not decide.  For each
 * qubit a = order[q], q = 0..k-1, in turn: rho_a of the current Vidal-gauge state gives the
 * outcome probabilities (p(+1) = rho_a[0,0]); the outcome is +1 if u[q] < rho_a[0,0], else -1;
 * Gamma_a is projected on that outcome (Eq. (projection)); then BP runs from the warm start
 * (tol, max_iter) and the network is regauged (App. D), as gtqa_bp_sweep with
 * GTQA_BP_DEFAULT does.  The state is left in its post-measurement form.
 *   k        number of qubits to sample (0 <= k <= n)
 *   order    int32 [k], host: distinct vertices
 *   u        float64 [k], host: the caller's uniform random numbers in [0, 1]
 *   x_out    int8 [n], host: +1 / -1 for the sampled qubits, 0 for the others
 *   p_out    float64 [k], host, nullable: the probability of each outcome given the earlier ones
 * For a batched state every step regauges all instances.  Synchronises the stream once (on a
 * plain-path state, see gtqa_create, also after every BP sweep).
 */
int gtqa_sample(gtqa_state* s, int32_t k, const int32_t* order, const double* u, double tol, int32_t max_iter,
                int8_t* x_out, double* p_out);

/*
 * Mean-field entanglement entropy of a bipartition (Sec. III C, Eq. (apprx_entropy) with the
 * Schmidt values of Eq. (mean_field_schmidt)): S* = - sum over the cut edges e of
 * sum_j lambda_e[j]^2 log(lambda_e[j]^2), computed on the device in FP64 from the current
 * lambda.
 *   cut    uint8 [m] (host or device): nonzero for the edges whose ends lie on different
 *          sides (for a batched state, m counts the edges of all instances)
 *   S_out  host double
 * Synchronises the stream.  GTQA_ERR_NUMERIC if the sum is NaN.
 */
int gtqa_entropy(gtqa_state* s, const uint8_t* cut, double* S_out);

/*
 * The bipartition of Eq. (bipartition), A* = argmin |dA| / (|A| |Abar|), by spectral
 * partitioning (host code): the eigenvector f of the second-smallest eigenvalue of the graph
 * Laplacian D - A (Lanczos with full reorthogonalisation on the complement of the constant
 * vector, at most 240 steps, so exact up to rounding for n <= 241; an approximation above),
 * its sign fixed so that its entry of largest modulus is positive, the vertices ordered by
 * (f, id), and the prefix of that order with the smallest ratio (the first one on ties).
 *   n, m, edges  the graph (int32 [m][2], host)
 *   side_out     uint8 [n], host: 1 for the vertices of A
 *   cut_out      uint8 [m], host, nullable: 1 for the edges between A and Abar
 *   ratio_out    host double, nullable: |dA| / (|A| |Abar|)
 * No device work.  GTQA_ERR_INVALID_ARG for n < 2 or an edge out of range or a self-loop.
 */
int gtqa_spectral_bipartition(int32_t n, int32_t m, const int32_t* edges, uint8_t* side_out, uint8_t* cut_out,
                              double* ratio_out);

/*
 * Residual of the local-orthogonality condition of the Vidal gauge (App. C, the distance to
 * the Vidal gauge): R = 1/(2|E|) sum_a sum_{b in da} || delta - sum Gamma_a Gamma_a^*
 * prod_{c != b} lambda_ca^2 ||_1 with the trace norm, computed in FP64 on the device from the
 * current Gamma and lambda.  delta is the identity on the bond indices with lambda > 0.
 *   R_out  host double, written on success (0 for a graph without edges)
 * Synchronises the stream.  GTQA_ERR_NUMERIC if the sum is NaN.
 */
int gtqa_residual(gtqa_state* s, double* R_out);

/*
 * Single-qubit reduced density matrices rho_a = sum Gamma Gamma^* prod_b lambda_ba^2 / tr
 * (Eq. (partial_dens) with the environment of Eq. (bp_approx) from the warm-start
 * messages of the current Vidal-gauge state) and the read-out of Eq. (rounding_rule).
 *   rho_out   complex128 [n][2][2] interleaved (host or device)
 *   sign_out  int8 [n] (+1 / -1), or NULL
 */
int gtqa_marginals(gtqa_state* s, double* rho_out, int8_t* sign_out);

/* Counters accumulated since creation (see gtqa_stats_t).  Synchronises the stream. */
int gtqa_stats(gtqa_state* s, gtqa_stats_t* out);

/*
 * Copy the state out (complex128 Gamma, float64 lambda, complex128 messages in the
 * layouts above; any pointer may be NULL to skip that array) or overwrite it (set:
 * every pointer required; lambda must be >= 0 and zero exactly beyond each bond's
 * dimension).  Used to start the library and a reference from identical states.
 * Messages are those of the last BP run, in the gauge that run saw: the gates and the
 * regauge change Gamma and lambda but not the messages.  In GTQA_MIXED the device holds
 * delta = m - diag(lambda)/sum(lambda) and get_state returns diag(lambda)/sum(lambda) + delta
 * with the current lambda; after gates or a regauge that sum is re-based on the new lambda
 * and is not the message of any BP run (the stale messages of the other modes are not
 * either).  A BP run without GTQA_BP_WARM_START continues from these values; runs with the
 * warm start (gtqa_anneal and the default flags) do not read them.
 */
int gtqa_get_state(gtqa_state* s, double* gamma_out, double* lambda_out, double* messages_out);
int gtqa_set_state(gtqa_state* s, const double* gamma, const double* lambda, const double* messages);

/* Number of bonds per vertex tensor: 3, or 4 for a graph with a degree-4 vertex (Gamma is
 * then [n][2][CHI][CHI][CHI][CHI] in gtqa_get_state / gtqa_set_state). */
int gtqa_max_degree(const gtqa_state* s, int32_t* D_out);

/* Sizes: total vertices and edges, storage bond dimension CHI, number of colours. */
int gtqa_sizes(const gtqa_state* s, int64_t* n, int64_t* m, int32_t* chi_storage, int32_t* n_colours);

/* Host-only: the edge colouring gtqa_create uses when colour is NULL: Delta colours by a
 * seeded Kempe-chain search when it succeeds (almost all random cubic graphs, trees,
 * heavy-hexagon lattices), else Misra-Gries (<= Delta + 1 colours).  Deterministic. */
int gtqa_edge_colouring(int32_t n, int32_t m, const int32_t* edges, int32_t* colour_out,
                        int32_t* n_colours_out);

/*
 * Optional profiler: with enable = 1 every launch is bracketed by CUDA events on the
 * state's stream (adds a little host overhead); enable = 0 stops recording.  Either
 * call clears the accumulated figures.
 */
int gtqa_profile(gtqa_state* s, int32_t enable);

/*
 * Accumulated figures of one kernel class (GTQA_K_*): launches, summed device time in
 * milliseconds (event pairs), and work units processed (edges for gate and regauge-edge
 * launches, vertices for vertex launches).  Synchronises the stream.
 */
int gtqa_profile_read(gtqa_state* s, int32_t kind, int64_t* launches, double* total_ms, int64_t* units);

/*
 * Test hook for the failure path of the bounded grid barriers: spin_limit sets the polls
 * a barrier waits before it gives up; extra_arrivals = 1 makes every barrier wait for one
 * block that does not exist, so the next launch returns GTQA_ERR_TIMEOUT (sticky) with the
 * device context intact.  Defaults: 4194304 polls, 0 extra arrivals.
 */
int gtqa_debug_barrier(gtqa_state* s, int64_t spin_limit, int32_t extra_arrivals);

/* Name of a launch class, or NULL if kind is out of range. */
const char* gtqa_profile_name(int32_t kind);

/*
 * Diagnostic: measured CUDA-core FMA throughput of the current device in TFLOP/s
 * (fp64 = 1: double, 0: float), the ALU roofline denominator for the arithmetic-bound
 * kernels.  Runs for a few milliseconds on the legacy default stream and synchronises.
 */
int gtqa_alu_peak(int32_t fp64, double* tflops_out);

/*
 * Diagnostic: for n positive host doubles x, writes 6 n host doubles: per x the kernels'
 * Newton-refined reciprocal, CUDA's 1/x, the refined 1/sqrt(x), CUDA's 1/sqrt(x), the
 * refined sqrt(x) and CUDA's sqrt(x) (accuracy tests of the divide-free arithmetic).
 */
int gtqa_math_check(int32_t n, const double* x, double* out);

/*
 * Diagnostic: average latency in microseconds of the bounded grid barrier that separates
 * the phases of the kernels (cooperative launch, one block of `threads` per SM, `rounds`
 * consecutive barriers, best of three launches).
 */
int gtqa_barrier_bench(int32_t threads, int32_t rounds, double* us_per_barrier);

/*
 * Belief propagation that allocates nothing (the paper has no counterpart; this is an
 * interface for callers that cannot allocate device memory here, e.g. latency-bound
 * loops that forbid cudaMalloc after start-up, or processes whose device memory belongs
 * to another allocator's pool).
 *
 * Runs the same flooding BP as gtqa_bp_sweep(tol, max_iter, GTQA_BP_WARM_START), FP64,
 * storage bond dimension GTQA_STATIC_CHI, on one instance held in caller-owned device
 * (or managed) memory:
 *   vert_edges    int32 [n][4]: edge id at bond slots 0..2 (-1 = phantom slot), degree
 *   edge_info     int32 [m][4]: u, v, slot of the edge in u, slot in v
 *                 (slots are a vertex's incident edges in ascending edge id)
 *   gamma         complex128 [n][2][4][4][4], Vidal-gauge tensors (read only)
 *   lambda        float64 [m][4], bond weights (read only)
 *   messages_out  complex128 [2m][4][4]: the final messages (row 2e = m_{u->v})
 *   iters_out, dist_out  nullable host pointers: sweeps run and final dist/|E|
 * Its scratch (symmetric-gauge tensors, second message buffer, control block) lives in a
 * file-scope device array of about 5.5 MiB that every GPU loading the library holds
 * until the process exits.  n > GTQA_STATIC_MAX_N or m > GTQA_STATIC_MAX_M, host
 * pointers, or bad sizes return GTQA_ERR_INVALID_ARG before any device work.  The
 * contents of vert_edges and edge_info are checked by a small kernel before BP runs
 * (degree 0..3, edge ids in [0, m), slots that agree between the two arrays, -1 past the
 * degree); a violation returns GTQA_ERR_INVALID_ARG and BP does not run.  Every call
 * looks up the array's device address (cudaGetSymbolAddress, which allocates nothing)
 * and sets the BP kernel's shared-memory limit, so calls remain valid after a device
 * reset.  All calls share the one array: calls that overlap on the GPU (other streams,
 * other threads) race.  Synchronises the stream.  Returns GTQA_ERR_NOT_CONVERGED when
 * max_iter was reached.
 */
#define GTQA_STATIC_CHI 4
#define GTQA_STATIC_MAX_N 2048
#define GTQA_STATIC_MAX_M 3072
int gtqa_bp_static(int32_t n, int32_t m, const int32_t* vert_edges, const int32_t* edge_info,
                   const double* gamma, const double* lambda, double* messages_out, double tol,
                   int32_t max_iter, int32_t* iters_out, double* dist_out, void* cuda_stream);

/* Static description of an error code. */
const char* gtqa_strerror(int code);

/* Release all device and host memory of s; NULL is allowed. */
void gtqa_destroy(gtqa_state* s);

#ifdef __cplusplus
}
#endif
#endif /* GTQA_H */
