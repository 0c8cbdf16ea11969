/*
 * msp.h -- C ABI of the GB300 synapse-search library (libmsp).
 *
 * The library computes, on one GPU, the structural-plasticity synapse search
 * of "Accelerating Brain Simulations with the Fast Multipole Method"
 * (Noettgen, Czappa, Wolf; arXiv 2301.10570):
 *
 *   u(t) = sum_{s != t} w_s exp(-|t - s|^2 / sigma^2)              (Eq. 8)
 *
 * for every neuron t with vacant axonal elements, where w_s is the number of
 * vacant dendritic elements of s of t's type.  The sum is organised on an
 * octree (Section 3.2) as a fast multipole method: Hermite coefficients of
 * source boxes (Eq. 7), their translation into Taylor coefficients about a
 * target box (Eq. 6), evaluation at the targets, and the exact near field.
 * The same pass yields the attraction between every pair of boxes the
 * descent of Algorithm 1 can visit; the descent then draws, per axon box and
 * level, a dendrite box with probability proportional to its attraction
 * (Algorithm 2) down to a dendrite neuron, and the requests are resolved at
 * the dendrite side (Section 4).
 *
 * Conventions (all entry points):
 *   - Every pointer named *_dev is a device pointer, *_host a host pointer.
 *     The caller owns every buffer it passes; the context owns its own
 *     workspace and frees it in msp_destroy.
 *   - Neuron arrays are in the caller's order (index 0..n-1); outputs are in
 *     the same order.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; the calls marked "synchronous" wait
 *     for it before returning.
 *   - Errors are returned as msp_status; msp_last_error() gives a message
 *     for the calling thread.  No call throws or aborts.
 *   - Channels: 0 = excitatory, 1 = inhibitory.  An axon of a type-T neuron
 *     connects only to vacant dendritic elements of channel T.
 *   - Results are deterministic for fixed inputs, configuration and step
 *     (every sum has a fixed order), except with centre_mode 1, whose grouped
 *     translations add into the Taylor coefficients atomically: there u may
 *     differ in the last bits between runs.
 */
#ifndef MSP_H
#define MSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct msp_ctx msp_ctx;

typedef enum {
    MSP_OK = 0,
    MSP_ERR_INVALID_ARG = 1,  /* bad pointer, size or configuration value    */
    MSP_ERR_CUDA = 2,         /* a CUDA runtime call failed                  */
    MSP_ERR_OOM = 3,          /* device allocation failed                    */
    MSP_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up          */
    MSP_ERR_NOT_BUILT = 5,    /* call order violated (e.g. no tree yet)      */
    MSP_ERR_CHECK = 6,        /* a device-side consistency check failed      */
    MSP_ERR_CAPACITY = 7      /* a size exceeds an index range (> 2^31-1)    */
} msp_status;

/* Search configuration.
 *   sigma          kernel width in the units of the positions (Table 1: 750)
 *   p              expansion terms per dimension, 1..8; multi-indices
 *                  0 <= alpha_d < p (the paper's alpha=beta=(3,3,3) is p=4)
 *   leaf_capacity  an octree box is split while it holds more points
 *   max_depth      deepest octree level, <= 21 (boxes at max_depth never split)
 *   origin, side   the cube [origin, origin+side)^3 quantised to 2^21 cells
 *                  per dimension; positions outside are clamped to its faces
 *   seed           Philox key of every random draw
 *   rho_max        an expansion is used only for boxes whose half-width is at
 *                  most rho_max*sigma
 *   cutoff         box pairs whose minimum distance is at least cutoff*sigma
 *                  contribute nothing (their kernel is below exp(-cutoff^2)),
 *                  and inside a chosen leaf sources beyond cutoff*sigma have
 *                  weight zero; 0 < cutoff <= 5 (exp(-25) ~ 1e-11 is below
 *                  single precision relative resolution of any sum)
 *   m2l_min_pairs  a well-separated pair is translated only if
 *                  count(X)*count(Y) >= m2l_min_pairs; otherwise it is
 *                  refined down to the near field
 *   centre_mode    expansion centres: 0 the weighted centroids (Section 3.2,
 *                  Section 4); 1 the boxes' geometric centres, for which a
 *                  translation depends only on the boxes' offset, so the
 *                  translations of all pairs with one offset run as one
 *                  matrix product (p <= 5)
 *   mac_mode       which box pairs are expanded: 0 (default) the accuracy
 *                  rule above (rho_max, separation, m2l_min_pairs); 1 the
 *                  paper's count rule of Algorithm 2: a pair of inner boxes
 *                  whose dendrite box holds more than c1 vacant dendritic
 *                  elements is expanded (Hermite when the axon box also holds
 *                  more than c2 vacant axonal elements, Taylor otherwise;
 *                  both run here as the one translation, Eq. 7 re-expanded by
 *                  Eq. 6), every other pair is refined to exact leaf pairs;
 *                  no size or distance criterion (every level may carry
 *                  expansions), the cutoff still prunes, a box is never
 *                  expanded against itself.  For comparison with the paper
 *                  (its expansions of boxes much wider than sigma are far
 *                  from the exact attraction); rho_max and m2l_min_pairs are
 *                  ignored in this mode
 *   c1, c2         Algorithm 2's thresholds (the paper: 70 and 70)           */
typedef struct {
    double    sigma;
    int       p;
    int       leaf_capacity;
    int       max_depth;
    float     origin[3];
    float     side;
    uint64_t  seed;
    double    rho_max;
    double    cutoff;
    long long m2l_min_pairs;
    int       centre_mode;
    int       mac_mode;
    int       c1, c2;
} msp_config;

/* Sizes and operation counts of the last build / attraction / selection. */
typedef struct {
    int64_t n;                 /* neurons                                   */
    int64_t n_nodes;           /* octree boxes                              */
    int64_t n_leaves;
    int32_t tree_depth;        /* deepest level present                     */
    int32_t far_level;         /* shallowest level allowed to carry expansions */
    int64_t n_pairs;           /* box pairs visited by the dual traversal   */
    int32_t pair_depths;
    int64_t n_far;             /* translated (M2L) pairs                    */
    int64_t n_p2p;             /* near-field leaf pairs                     */
    int64_t p2p_interactions;  /* target-source evaluations in the near field */
    int64_t n_elements;        /* vacant axonal elements (sum of vac_axon)  */
    int64_t n_draws;           /* tree-level + leaf draws of the last selection */
    int64_t n_requests;        /* elements that drew a partner              */
    int64_t n_synapses;        /* accepted requests                         */
    int64_t expansion_nodes;   /* boxes carrying expansions                 */
    int64_t kernel_launches;   /* kernels launched by this library in this
                                  process so far (all contexts)             */
    double  near_field_ms;     /* device time of the near-field kernel of the
                                  last msp_attraction (CUDA events on its
                                  stream); 0 if it had no near-field pairs  */
} msp_stats;

/* Create a context on CUDA device `device` (cudaSetDevice is called).
 * Ownership: the caller destroys it with msp_destroy.  Errors:
 * MSP_ERR_INVALID_ARG for a configuration outside the ranges above. */
msp_status msp_create(msp_ctx **out, const msp_config *cfg, int device);
msp_status msp_destroy(msp_ctx *ctx);

/* Steps a1-a4 (Section 3.2): Morton keys of the positions, a stable radix
 * sort, the adaptive octree (level by level; a box with more than
 * leaf_capacity points is split into its non-empty octants) and, per box,
 * the sums of vacant axonal elements per channel, vacant dendritic elements
 * per channel, and the axon- and dendrite-weighted centroids.
 *   x_dev,y_dev,z_dev    n floats each (SoA positions)
 *   type_dev             n bytes, 0/1
 *   vac_axon_dev         n bytes, vacant axonal elements of the neuron's type
 *   vac_dend_e_dev/_i    n bytes, vacant dendritic elements per channel
 * The inputs are read during the call's stream work only; the context keeps
 * its own sorted copy.  The octree depends on the positions only: when n and
 * the positions equal those of the context's last build (a checksum of every
 * coordinate's bits, read back: one more synchronisation), the sorted order
 * and the octree are kept and only the counts and aggregates are refreshed.
 * Synchronous (the per-level node counts are read back).  n may be 0.  Errors: MSP_ERR_INVALID_ARG (n < 0, n > 2^31-2, null
 * pointer with n > 0, a position outside [origin, origin + side) or not
 * finite: the boxes of the tree must contain their points), MSP_ERR_OOM
 * (including the workspace limit of msp_set_workspace_limit). */
msp_status msp_build_tree(msp_ctx *ctx, int64_t n, const float *x_dev, const float *y_dev,
                          const float *z_dev, const uint8_t *type_dev,
                          const uint8_t *vac_axon_dev, const uint8_t *vac_dend_e_dev,
                          const uint8_t *vac_dend_i_dev, void *stream);

/* Steps a5-a10: dual traversal (Algorithm 1's pairing of axon and dendrite
 * boxes, refined until a pair is pruned by the cutoff, translated, or a
 * near-field leaf pair), Hermite coefficients (Eq. 7), Hermite-to-Taylor
 * translation (composition of Eq. 7 and Eq. 6), Taylor evaluation (Eq. 6),
 * exact near field (Eq. 8), and the box-pair attraction table.
 *   u_dev   n floats out: u(t) of the neuron's own channel if vac_axon > 0,
 *           else 0.  May be NULL (only the pair table is produced).
 * The traversal prunes by the cutoff only (mac_mode 0), so its interaction
 * lists depend on the positions and the kernel width alone: after a build
 * that kept the octree, the lists of the last attraction are kept as well
 * (the counts, expansions, near field and pair table are recomputed).
 * Requires msp_build_tree.  Synchronous (per-depth pair counts are read
 * back).  Errors: MSP_ERR_NOT_BUILT, MSP_ERR_OOM, MSP_ERR_CAPACITY. */
msp_status msp_attraction(msp_ctx *ctx, float *u_dev, void *stream);

/* The comparison path: Eq. 8 by all-pairs evaluation over every neuron, on
 * the tree's sorted copy (no cutoff, no expansion).  Same output convention
 * as msp_attraction.  Requires msp_build_tree.  Asynchronous. */
msp_status msp_direct(msp_ctx *ctx, float *u_dev, void *stream);

/* Steps a11-a12: Algorithm 1 with Algorithm 2's choice at every level, a
 * per-element draw inside the chosen dendrite leaf, and request resolution.
 * The level draws take prefix sums of the candidates' attractions in pairs
 * of floats (hi + lo), the leaf draw in exact 64-bit fixed point; a dendrite
 * neuron accepts, per channel, its first requests in (Philox priority,
 * element) order up to its vacant count.
 *   step            plasticity step number, part of every Philox counter
 *   partner_dev     n_elements int32 out: the dendrite neuron drawn by each
 *                   vacant axonal element (elements ordered by neuron, then
 *                   element index; n_elements = sum of vac_axon), -1 if none
 *   syn_pre_dev, syn_post_dev (int32), syn_type_dev (uint8): capacity
 *                   n_elements; the accepted synapses in element order
 *   n_syn_dev       one int64 out: number of synapses written
 * Requires msp_attraction.  Synchronous.  Errors: MSP_ERR_NOT_BUILT. */
msp_status msp_select_partners(msp_ctx *ctx, uint64_t step, int32_t *partner_dev,
                               int32_t *syn_pre_dev, int32_t *syn_post_dev,
                               uint8_t *syn_type_dev, int64_t *n_syn_dev, void *stream);

/* One whole plasticity step (steps a1-a12: build + attraction + selection)
 * from HOST buffers: copies the inputs to the context's device staging
 * buffers, runs the path, and copies u, partner and the synapse list back.
 * Host buffers should be pinned for full copy bandwidth.  partner_host and
 * syn_* have capacity sum(vac_axon).  u_host may be NULL.  Returns the synapse
 * count in *n_syn_host.  The results equal those of msp_build_tree,
 * msp_attraction and msp_select_partners on the same inputs.
 * The first call runs the path as separate kernels and then captures it as a
 * CUDA graph on the staging buffers (the context's second graph, apart from
 * msp_step_graph_*); later calls with the same n replay that graph, which
 * reuses the octree while the positions equal those of the capture (a
 * checksum of the positions is compared on the device) and refreshes its
 * counts and aggregates.  A call the graph cannot serve (another n, changed
 * positions, more vacant elements than it holds, a workspace reallocated by
 * another call) runs eagerly and captures again.  Two host synchronisations
 * per replayed call: the step's sizes, then the copies back.  Runs on the
 * legacy default stream.  Synchronous. */
msp_status msp_plasticity_step_host(msp_ctx *ctx, int64_t n, uint64_t step,
                                    const float *x_host, const float *y_host,
                                    const float *z_host, const uint8_t *type_host,
                                    const uint8_t *vac_axon_host,
                                    const uint8_t *vac_dend_e_host,
                                    const uint8_t *vac_dend_i_host, float *u_host,
                                    int32_t *partner_host, int32_t *syn_pre_host,
                                    int32_t *syn_post_host, uint8_t *syn_type_host,
                                    int64_t *n_syn_host);

/* Vacancy random walk used by the 100-step clustered run: every neuron's
 * vacant axonal and dendritic counts move by +1 or -1 (Philox, tag WALK,
 * counter (neuron, channel, step)), clamped to [0,5].  In place, n bytes
 * each.  Asynchronous. */
msp_status msp_vacancy_walk(msp_ctx *ctx, int64_t n, uint64_t step, uint8_t *vac_axon_dev,
                            uint8_t *vac_dend_e_dev, uint8_t *vac_dend_i_dev, void *stream);

/* Formed synapses occupy their elements (Section 3.1: vacant = elements -
 * synapses): decrement vac_axon of each pre neuron and the dendritic count
 * of the synapse's channel of each post neuron, saturating at 0.
 * n_syn_dev is read on the device.  Asynchronous. */
msp_status msp_commit_synapses(msp_ctx *ctx, const int64_t *n_syn_dev, int64_t capacity,
                               const int32_t *syn_pre_dev, const int32_t *syn_post_dev,
                               const uint8_t *syn_type_dev, uint8_t *vac_axon_dev,
                               uint8_t *vac_dend_e_dev, uint8_t *vac_dend_i_dev,
                               void *stream);

/* Self-test of the device's bounded waits: runs the single-pass scan with a
 * predecessor tile that never publishes its sum, so the waiting tiles give
 * up after a bounded number of polls.  Returns MSP_ERR_TIMEOUT when the wait
 * gave up as designed (any other status is a failure); the context stays
 * usable.  Synchronises. */
msp_status msp_selftest_bounded_wait(msp_ctx *ctx, void *stream);

/* ---- The neuron side of the model (Section 3.1, Table 1) -------------------
 * The Model of Structural Plasticity's neurons produce the vacant elements
 * that the synapse search consumes.  The network's synapses are an edge list
 * (pre, post, type) in caller-owned device memory, in insertion order, with
 * its length in device memory (*n_edges_dev) and a capacity; type = the
 * channel (the pre neuron's type).  Every edge must name neurons in [0, n).
 * The neuron state is caller-owned device memory, n entries each: activity x,
 * refractory counter, calcium, the element counts z (continuous) of the axon
 * and of the two dendrite types, and last step's spike flags.  Draws use the
 * context's seed.  All three calls are bit-for-bit reproducible. */
typedef struct {
    float x0;              /* resting potential (Table 1: 0.05)             */
    float tau_x;           /* membrane potential decay constant (5)         */
    float background;      /* background activity per step (0.003)          */
    float input_per_spike; /* per synapse from a neuron that spiked (5e-4)  */
    int   refractory;      /* steps without a spike after one (4), <= 255   */
    float beta_ca;         /* calcium increase per spike (5e-4)             */
    float decay_ca;        /* calcium decay per step (1e-5)                 */
    float eps;             /* growth curve right intersection (0.7)         */
    float eta_axon;        /* growth curve left intersection, axons (0.4)   */
    float eta_dend;        /* left intersection, dendrites (0.1)            */
    float mu;              /* growth scaling, the maximum rate (1e-4)       */
} msp_neuron_params;

/* n_steps simulation steps first_step .. first_step + n_steps - 1 (Section
 * 3.1).  Per step and neuron t: input = number of edges s -> t whose s
 * spiked in the previous step (spiked_dev on entry); x <- x + (x0 - x)/tau_x
 * + background + input_per_spike * input; unless refractory, a Philox draw
 * U in [0,1) fires when U < x (then refractory = `refractory`); calcium
 * decays by decay_ca and rises by beta_ca on a spike; each z grows by the
 * Gaussian growth curve mu (2 exp(-((Ca - xi)/zeta)^2) - 1), xi = (eta +
 * eps)/2, zeta = (eps - eta)/(2 sqrt(ln 2)) (eta_axon for the axon, eta_dend
 * for both dendrites), and stays >= 0.  Single precision.  At most
 * edge_capacity edges are read; an edge naming a neuron outside [0, n) is
 * skipped.  Asynchronous. */
msp_status msp_neuron_steps(msp_ctx *ctx, int64_t n, uint64_t first_step, int n_steps,
                            const msp_neuron_params *params, const int64_t *n_edges_dev,
                            int64_t edge_capacity, const int32_t *edge_pre_dev,
                            const int32_t *edge_post_dev,
                            float *x_dev, uint8_t *refractory_dev, float *calcium_dev,
                            float *z_axon_dev, float *z_dend_e_dev, float *z_dend_i_dev,
                            uint8_t *spiked_dev, void *stream);

/* Update of synapses (Section 3.1): a neuron with more bound synapses on a
 * side (outgoing; incoming of each type) than floor(z) deletes the excess,
 * chosen uniformly at random with Philox step `step`; an edge chosen by
 * either of its sides is removed and the list compacted in place, order
 * kept.  Then vac = clamp(floor(z) - bound, 0, 255) for the axon and both
 * dendrite types.  Synchronises once (it checks the edges: an endpoint
 * outside [0, n) gives MSP_ERR_INVALID_ARG and changes nothing). */
msp_status msp_update_synapses(msp_ctx *ctx, int64_t n, uint64_t step, const float *z_axon_dev,
                               const float *z_dend_e_dev, const float *z_dend_i_dev,
                               int64_t *n_edges_dev, int32_t *edge_pre_dev,
                               int32_t *edge_post_dev, uint8_t *edge_type_dev,
                               int64_t edge_capacity, uint8_t *vac_axon_dev,
                               uint8_t *vac_dend_e_dev, uint8_t *vac_dend_i_dev, void *stream);

/* Append the synapses formed by msp_select_partners (*n_syn_dev of them, at
 * most syn_capacity, the length of the syn_* arrays) to the edge list.  Synchronises once; when the capacity is exceeded, the
 * synapses that fit are appended and MSP_ERR_CAPACITY is returned. */
msp_status msp_append_synapses(msp_ctx *ctx, const int64_t *n_syn_dev, int64_t syn_capacity,
                               const int32_t *syn_pre_dev, const int32_t *syn_post_dev,
                               const uint8_t *syn_type_dev, int64_t *n_edges_dev, int32_t *edge_pre_dev,
                               int32_t *edge_post_dev, uint8_t *edge_type_dev,
                               int64_t edge_capacity, void *stream);

/* ---- The whole plasticity step as one CUDA graph ---------------------------
 * A plasticity step of the 100-step run is: vacancy walk (step k), octree
 * build (Section 3.2), attraction (Section 3.3, Eq. 6-8), selection
 * (Algorithm 1, Algorithm 2, Section 4) with Philox step k, commit of the
 * formed synapses.  msp_step_graph_capture records that sequence once, on
 * the device buffers given, as a CUDA graph; msp_step_graph_launch replays
 * it, one replay per step, with the step index kept and advanced in device
 * memory, so a run of many steps needs no host work per step.
 *
 * Capture requirements: msp_build_tree and msp_attraction have run on the
 * same positions x/y/z (their tree depth and pair-table size give the
 * graph's capacities).  Unless the full-build option is set, the replays
 * keep that build's octree and that attraction's traversal and pair lists
 * (they depend on the positions only, for mac_mode 0) and redo the counts,
 * aggregates, expansions, near field, pair table and everything after.  The positions and types must not change while the
 * graph is in use (neurons do not move in the model); the vacant counts are
 * the run's state, changed only by the graph (walk and commit).
 *   x/y/z/type_dev     n neurons, read every replay
 *   vac_*_dev          the state, updated in place every replay
 *   partner_dev        capacity 5*n int32 (the walk keeps counts <= 5)
 *   syn_*_dev          capacity syn_capacity >= 5*n
 *   n_syn_dev          one int64: the last replay's synapse count
 *   history_dev        optional (NULL): int64[history_len], entry i receives
 *                      the synapse count of step first_step + i
 *   first_step         the step index of the first replay
 * The capture runs one dry pass (nothing of the state changes) to size the
 * workspace, then records; it synchronises `stream`.
 *
 * A replay that would exceed a capacity (pair table, descent items, tree
 * depth) sets a device-side halt flag before its commit; that step's and all
 * later replays' walk and commit then change nothing.  msp_step_graph_finish
 * waits for the replays, finishes a halted step eagerly (growing what
 * overflowed), captures the graph again from the next step, and returns the
 * index of the next step to run in *next_step (so the caller replays the
 * remaining steps) and the halt bits in *halted (0: none).
 * Errors: MSP_ERR_NOT_BUILT (capture before build/attraction, launch without
 * a graph), MSP_ERR_INVALID_ARG. */
msp_status msp_step_graph_capture(msp_ctx *ctx, int64_t n, const float *x_dev,
                                  const float *y_dev, const float *z_dev,
                                  const uint8_t *type_dev, uint8_t *vac_axon_dev,
                                  uint8_t *vac_dend_e_dev, uint8_t *vac_dend_i_dev,
                                  int32_t *partner_dev, int32_t *syn_pre_dev,
                                  int32_t *syn_post_dev, uint8_t *syn_type_dev,
                                  int64_t syn_capacity, int64_t *n_syn_dev,
                                  int64_t *history_dev, int64_t history_len,
                                  uint64_t first_step, void *stream);
/* Option of the next msp_step_graph_capture: full_build = 1 makes every
 * replay rebuild the octree from the positions (Morton keys, radix sort,
 * subdivision, aggregates: steps a1-a4 in full); 0 (the default) reuses the
 * octree of the eager build and refreshes its counts and aggregates, checked
 * on the device by a checksum of the positions and the build's generation
 * stamp (a mismatch halts the replay, see above).  Both give the same
 * results while the positions are unchanged. */
msp_status msp_step_graph_set_full_build(msp_ctx *ctx, int full_build);

/* Enqueues n_steps replays on `stream`.  Asynchronous.  Fails with
 * MSP_ERR_NOT_BUILT if any workspace buffer of the library was reallocated
 * since the capture (an eager call on larger inputs): capture again. */
msp_status msp_step_graph_launch(msp_ctx *ctx, int64_t n_steps, void *stream);
/* Waits for the replays (see above).  msp_get_stats then reports the last
 * replay's sizes and, in near_field_ms and p2p_interactions, the means over
 * the replays of the last launch.  Synchronous. */
msp_status msp_step_graph_finish(msp_ctx *ctx, void *stream, uint64_t *next_step,
                                 int64_t *halted);
/* Capacity of the pair table (box pairs of the dual traversal).  The table
 * grows on demand in the eager calls; inside the step graph it cannot, and a
 * step that needs more halts (see above).  Values below the current use are
 * allowed (the next eager attraction grows the table again). */
msp_status msp_set_pair_capacity(msp_ctx *ctx, int64_t pairs);

/* ---- Derivatives of the attraction (the adjoint of Eq. 8) -----------------
 * With K(t,s) = exp(-|t - s|^2 / sigma^2), at the counts given here (DEVICE,
 * caller order, n = the last build's neurons):
 *   u(t)          = sum_{s != t} w_s^{T(t)} K(t,s)              (a_t > 0, else 0)
 *   du_dsigma(t)  = sum_{s != t} w_s^{T(t)} K(t,s) 2 |t - s|^2 / sigma^3
 *   grad_w_e(s), grad_w_i(s) = sum_{t != s, a_t > 0, T(t) = E resp. I} g_t K(t,s),
 * i.e. the gradient of L = sum_t g_t u(t) with respect to the dendritic
 * weights w^E, w^I (the transposed Gauss transform; dL/dsigma is
 * sum_t g_t du_dsigma(t)).  The sums run over the near-field leaf pairs of
 * the last msp_attraction, which must have no translated pairs
 * (rho_max = 0).  The lists depend on the positions only (no box pair is
 * dropped for empty counts), so the derivatives with respect to weights that
 * are zero are complete; the counts passed here are the ones the derivatives
 * are taken at.  g may be NULL (then
 * grad_w_* must be NULL); any output may be NULL.  Errors: MSP_ERR_NOT_BUILT,
 * MSP_ERR_INVALID_ARG (translated pairs present).  Asynchronous. */
msp_status msp_attraction_grad(msp_ctx *ctx, const uint8_t *type_dev,
                               const uint8_t *vac_axon_dev, const uint8_t *vac_dend_e_dev,
                               const uint8_t *vac_dend_i_dev, const float *g_dev, float *u_dev,
                               float *du_dsigma_dev, float *grad_w_e_dev, float *grad_w_i_dev,
                               void *stream);

/* ---- Expected mean synapse length and its gradient ------------------------
 * The calibration target of the differentiation workload.  An axonal element
 * of t draws dendrite s with probability w_s K(t,s) / u(t) (Eq. 1 with the
 * kernel of Eq. 8, K = exp(-|t - s|^2 / sigma^2); w the continuous dendritic
 * weights of t's channel), so its synapse is on average
 *   l(t) = v(t) / u(t) long,  u(t) = sum_s w_s K,  v(t) = sum_s w_s K |t - s|.
 * Over the vacant axonal elements (a_t > 0, u(t) > 0):
 *   m = sum_t a_t l(t) / sum_t a_t,   loss = (m - target)^2.
 *   type_dev, vac_axon_dev   n bytes (caller order): channels and a_t
 *   w_e_dev, w_i_dev         n floats: dendritic weights per channel
 *   out4_host                4 doubles out: loss, m, dloss/dsigma, dm/dsigma
 *   grad_w_e_dev/_i_dev      n floats out (either may be NULL): dloss/dw^E,
 *                            dloss/dw^I (the transposed sums; K is symmetric)
 * The sums run over the near-field leaf pairs of the last msp_attraction,
 * which must have no translated pairs (|t - s| has no Hermite expansion);
 * use a cutoff of 5 (the sums then miss terms below exp(-25)).
 * Single precision sums with Kahan-compensated chunks; the scalar reductions
 * in double, in a fixed order (reproducible).  Errors: MSP_ERR_NOT_BUILT,
 * MSP_ERR_INVALID_ARG (translated pairs present).  Synchronous. */
msp_status msp_length_loss(msp_ctx *ctx, const uint8_t *type_dev, const uint8_t *vac_axon_dev,
                           const float *w_e_dev, const float *w_i_dev, double target,
                           double *out4_host, float *grad_w_e_dev, float *grad_w_i_dev,
                           void *stream);

/* Sets the kernel width sigma of the context (the rest of the configuration
 * stays).  The octree stays (it depends on the positions only); the pair
 * lists and the pair table depend on sigma (cutoff radius, expansion
 * boxes), so msp_attraction must run again before the calls that need it,
 * and captured step graphs are released.  For the calibration of sigma
 * against a target mean synapse length.  Errors: MSP_ERR_INVALID_ARG. */
msp_status msp_set_sigma(msp_ctx *ctx, double sigma);

/* Cap on the device memory that the workspaces of all contexts of this
 * process may hold (bytes; 0, the default, means none).  A workspace
 * allocation beyond it fails with MSP_ERR_OOM and leaves the context usable
 * (for processes that share a GPU, and to exercise the out-of-memory path).
 * Does not free memory already held: destroy contexts for that.  Applies to
 * allocations after the call. */
msp_status msp_set_workspace_limit(int64_t bytes);
/* Device memory held by the workspaces of all contexts of this process. */
int64_t msp_workspace_bytes(void);

/* Sizes and counts of the last calls.  Synchronous. */
msp_status msp_get_stats(msp_ctx *ctx, msp_stats *out);

/* Copies of internal arrays for parity tests (all HOST pointers, sizes from
 * msp_get_stats; any pointer may be NULL to skip that array).  Synchronous.
 *   keys (n uint64, sorted Morton keys), perm (n int32, caller index of each
 *   sorted position); per box: level, prefix (Morton code at its level),
 *   first, count, parent, child_first (-1 for a leaf), nchild,
 *   sums4 (n_nodes x {axon E, axon I, dendrite E, dendrite I}),
 *   cent6 (n_nodes x {axon centroid xyz, dendrite centroid xyz}). */
msp_status msp_export_tree(msp_ctx *ctx, uint64_t *keys, int32_t *perm, uint8_t *level,
                           uint64_t *prefix, int32_t *first, int32_t *count, int32_t *parent,
                           int32_t *child_first, uint8_t *nchild, int32_t *sums4,
                           float *cent6);

/* Box pairs of the dual traversal (HOST pointers, n_pairs each; depth_start
 * has pair_depths+1 entries): kind 0 split, 1 far (translated), 2 near-field
 * leaf pair, 3 pruned; w_e / w_i the pair attraction per channel (the
 * device table holds each as a pair of floats hi + lo, about 48 significant
 * bits, summed here in double). */
msp_status msp_export_pairs(msp_ctx *ctx, int32_t *X, int32_t *Y, uint8_t *kind,
                            int32_t *child_first, double *w_e, double *w_i,
                            int64_t *depth_start);

/* Expansions of the boxes at level >= far_level, HOST float arrays of
 * expansion_nodes x 2 x p^3 each (channel-major): A (Hermite coefficients of
 * the dendritic weights), M (axon moments), B (accumulated Taylor
 * coefficients); first_node receives the index of the first such box. */
msp_status msp_export_expansions(msp_ctx *ctx, float *A, float *M, float *B,
                                 int64_t *first_node);

/* Message of the last error of the calling thread ("" if none). */
const char *msp_last_error(void);

/* ---- Many independent networks as one problem (batched step) ------------
 * The attraction depends on positions only through |t - s| / sigma, so a
 * network scaled by 1/sigma has kernel width 1.  msp_batch_layout scales each
 * network k (neurons [offsets[k], offsets[k+1]) of the concatenated arrays,
 * kernel width sigma[k]) by 1/sigma[k] and gives it its own cell of a grid of
 * octree boxes at level *level_out, on every other cell of each dimension
 * (cell k at grid coordinates 2 (k mod G, (k / G) mod G, k / G^2),
 * G = 2^(level-1)), so any two networks are more than `cutoff` apart.  The
 * positions it writes are each network's own, relative to the low corner of
 * its cell: a context created with sigma = 1, origin = 0, side = *side_out
 * and the same cutoff and leaf capacity, and told of the frames by
 * msp_set_frames(ctx, n_networks, offsets, *level_out), then runs the whole
 * batch through the ordinary calls (or the step graph) in one pass.  Box
 * pairs between networks are pruned exactly, and every leaf and every shared
 * axon-box choice of Algorithm 1 lies inside one network (each network has
 * more neurons than the leaf capacity, so every box above its cell is split).
 * Neuron order is unchanged: u, partner and synapse indices refer to the
 * concatenated arrays.  The cell side is a power of two (the widest scaled
 * network plus cutoff + 1, rounded up).
 *   offsets            HOST, n_networks + 1 int64, offsets[0] = 0
 *   x,y,z              DEVICE, offsets[n_networks] positions (any unit)
 *   sigma              HOST, n_networks kernel widths (same unit)
 *   x_out,y_out,z_out  DEVICE, the scaled positions (sigma units) relative to
 *                      the network's cell, in [0, side_out / 2^level_out)
 *   side_out, level_out HOST: the domain side and the level of the cells
 * Errors: MSP_ERR_INVALID_ARG (a network with <= leaf_capacity neurons,
 * sigma <= 0, non-finite positions, bad offsets).  Needs no context;
 * allocates a few bytes per network of device scratch.  Synchronous. */
msp_status msp_batch_layout(int64_t n_networks, const int64_t *offsets, const float *x_dev,
                            const float *y_dev, const float *z_dev, const double *sigma,
                            double cutoff, int leaf_capacity, float *x_out_dev,
                            float *y_out_dev, float *z_out_dev, float *side_out,
                            int *level_out, void *stream);

/* Independent networks in their own frames (the batched step of
 * msp_batch_layout).  Network k holds the caller-order neurons
 * [offsets[k], offsets[k+1]); its positions are given relative to the low
 * corner of its cell of the octree grid at `level` (side / 2^level wide), the
 * cell at grid coordinates 2 (k mod G, (k / G) mod G, k / G^2), G =
 * 2^(level-1), and lie in [0, side / 2^level).  The Morton key of a point
 * holds its cell in the top `level` bits of each axis and its local position
 * below them, so the octree, the pair lists and every draw are those of the
 * networks side by side in one domain; but positions, box centres and
 * centroids stay in each network's own frame, so single precision keeps a
 * network's own resolution however wide the batch's domain.  Boxes above the
 * cell level span several networks: they carry no expansion and are never
 * translated (mac_mode 1 included).  msp_direct takes, for each target, the
 * sources of its own network only.  n_networks = 0 removes the frames.
 * Per-network plans: leaf_capacity[k] and cutoff[k] (either may be NULL: the
 * configuration's value for every network) replace the configuration's leaf
 * capacity and cutoff inside network k: its boxes split above its own
 * capacity, its box pairs are pruned at its own cutoff, and its leaf draws
 * are truncated at its own radius (boxes above the cell level always split
 * and are pruned at the largest cutoff).
 *   offsets  HOST, n_networks + 1 int64: offsets[0] = 0, every network with
 *            more neurons than the leaf capacity; the next msp_build_tree
 *            must be given offsets[n_networks] neurons
 *   level    1..min(10, max_depth - 1); n_networks <= G^3; side / 2^level
 *            must exceed every cutoff * sigma
 *   leaf_capacity  HOST, n_networks int32 >= 1 (each network larger), or NULL
 *   cutoff         HOST, n_networks doubles in (0, 5], or NULL
 * The context's octree, pair lists and captured step graphs are dropped.
 * Errors: MSP_ERR_INVALID_ARG; a position outside its cell makes the next
 * msp_build_tree fail with MSP_ERR_INVALID_ARG.  Synchronous. */
msp_status msp_set_frames(msp_ctx *ctx, int64_t n_networks, const int64_t *offsets, int level,
                          const int32_t *leaf_capacity, const double *cutoff);

/* The counter-based generator behind every random draw of the library:
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11), ten rounds, run on the device for n caller-given
 * counters and keys, so that a caller can check the stream the draws use
 * against the published known-answer vectors.  The draws of the search use
 * key = (seed_lo, seed_hi) and counter = (c0, c1, step_lo, step_hi) with
 * U = top 53 bits of output words 0 and 1.
 *   ctr   DEVICE, n x 4 uint32 counters
 *   key   DEVICE, n x 2 uint32 keys
 *   out   DEVICE, n x 4 uint32 output blocks
 * Needs no context.  Errors: MSP_ERR_INVALID_ARG (n < 0, null pointer with
 * n > 0).  Asynchronous on `stream`. */
msp_status msp_philox(int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out,
                      void *stream);

/* Largest n accepted by msp_direct_noalloc (the size of its fixed scratch). */
#define MSP_NOALLOC_MAX_N 65536

/* The all-pairs attraction of msp_direct for callers that cannot allocate
 * device memory: a simulation loop that must never block on cudaMalloc (which
 * can synchronise the device), or a host framework that owns all device
 * memory and forbids libraries to allocate.  The paper has no counterpart;
 * this is a service of this library.
 *   n                    number of neurons, 0..MSP_NOALLOC_MAX_N; larger n is
 *                        rejected with MSP_ERR_INVALID_ARG and nothing runs
 *   x,y,z,type,vac_*     device inputs as for msp_build_tree (caller order)
 *   sigma                kernel width
 *   u                    device output, n floats: u(t) of the neuron's own
 *                        channel if vac_axon > 0, else 0
 *   stream               cudaStream_t as void* (NULL = legacy default stream)
 * It allocates nothing and needs no context.  Its scratch is one fixed
 * file-scope device array of MSP_NOALLOC_MAX_N * 24 bytes that every GPU
 * loading this library holds until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with the
 * device current; make that first call before any stream capture.  The
 * address is kept per device and CUDA context: after cudaDeviceReset (a new
 * context) the next call looks it up again, so that call, too, belongs before
 * any stream capture.  Every pointer must be device (or managed) memory of
 * the current device; others give MSP_ERR_INVALID_ARG.  All calls
 * share the array and it keeps the last call's contents (each call rewrites
 * the part it reads before reading it), so calls whose work overlaps on the
 * same GPU (for example on two streams) race on it: the caller must
 * serialise them.  Asynchronous on `stream`. */
msp_status msp_direct_noalloc(int64_t n, const float *x, const float *y, const float *z,
                              const uint8_t *type, const uint8_t *vac_axon,
                              const uint8_t *vac_dend_e, const uint8_t *vac_dend_i,
                              double sigma, float *u, void *stream);

#ifdef __cplusplus
}
#endif
#endif
