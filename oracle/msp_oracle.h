/*
 * msp_oracle.h -- plain FP64 CPU oracle for the FMM synapse search of
 * "Accelerating Brain Simulations with the Fast Multipole Method"
 * (Noettgen, Czappa, Wolf; arXiv 2301.10570).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library
 * against an obviously correct, slow restatement of the method.  Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header or table with the CUDA path.
 *
 * Every floating-point quantity is double precision, except the Morton
 * quantisation, which is done in single precision with round-to-nearest so
 * that the integer keys (and hence the tree) are the same on both sides.
 *
 * The Philox stream is pinned by the generator's published known-answer
 * vectors (Salmon et al., SC'11).
 */
#ifndef MSP_ORACLE_H
#define MSP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Configuration of one synapse search.  sigma: width of the Gaussian
 * attraction exp(-|t-s|^2 / sigma^2) (Eq. 8).  p: expansion terms per
 * dimension (multi-indices 0 <= alpha_d < p, the truncation of Eq. 6/7).
 * leaf_capacity, max_depth: octree leaves hold at most leaf_capacity points
 * unless they sit at max_depth (Section 3.2).  origin/side: the cube that is
 * quantised into the 2^21 Morton grid.  rho_max: largest box half-width, in
 * units of sigma, allowed to carry an expansion.  cutoff: box pairs whose
 * minimum distance is at least cutoff*sigma are dropped.  m2l_min_pairs:
 * a box pair is translated only when count_X * count_Y reaches this. */
typedef struct {
    double   sigma;
    int      p;
    int      leaf_capacity;
    int      max_depth;
    float    origin[3];
    float    side;
    uint64_t seed;
    double   rho_max;
    double   cutoff;
    long long m2l_min_pairs;
    double   boundary_tol;   /* draws within this relative distance of a CDF
                                boundary are flagged (not an algorithm input) */
    int      centre_mode;    /* expansion centres: 0 the weighted centroids
                                (Section 3.2, Section 4), 1 the boxes'
                                geometric centres */
    int      mac_mode;       /* 1: Algorithm 2's count rule chooses the
                                expanded pairs (c1 dendrites; c2 would pick
                                Hermite over Taylor, one translation here) */
    int      c1, c2;
} orc_config;

typedef struct orc_ctx orc_ctx;

/* pair kinds of the dual traversal */
enum { ORC_SPLIT = 0, ORC_FAR = 1, ORC_P2P = 2, ORC_PRUNED = 3 };

orc_ctx *orc_create(const orc_config *cfg);
void     orc_destroy(orc_ctx *c);

/* Step a1-a4: Morton keys, stable sort, adaptive octree, box aggregates. */
int orc_build_tree(orc_ctx *c, int64_t n, const float *x, const float *y,
                   const float *z, const uint8_t *type, const uint8_t *vac_axon,
                   const uint8_t *vac_dend_e, const uint8_t *vac_dend_i);

/* Step a5-a10: dual traversal, P2M, M2L, L2P, P2P, pair-table reduction.
 * u[i] = attraction of neuron i's own channel if vac_axon[i] > 0, else 0. */
int orc_attraction(orc_ctx *c, double *u);

/* Step a11-a12: descent + leaf draw + request resolution.
 * partner: one entry per vacant axonal element, elements ordered by neuron
 * then element index; -1 where no partner was drawn.  near_boundary: 1 where
 * some draw on the element's path fell within boundary_tol of a CDF edge.
 * accepted: 1 where the request was accepted.  Returns the synapse count. */
int64_t orc_select_partners(orc_ctx *c, uint64_t step, int32_t *partner,
                            uint8_t *near_boundary, uint8_t *accepted,
                            int32_t *syn_pre, int32_t *syn_post, uint8_t *syn_type);

/* Exact attraction by brute force over all sources (Eq. 8), for the listed
 * targets.  Same convention as orc_attraction's u. */
void orc_direct(int64_t n, const float *x, const float *y, const float *z,
                const uint8_t *type, const uint8_t *vac_axon,
                const uint8_t *vac_dend_e, const uint8_t *vac_dend_i,
                double sigma, int64_t n_targets, const int64_t *targets,
                double *u);

/* Derivatives of the attraction (Eq. 8, K = exp(-r^2/sigma^2)), all arrays
 * in caller order, evaluated at the counts given here:
 *   u(t)         = sum_{s != t} w_s^{T(t)} K(t,s)             (a_t > 0, else 0)
 *   dudsig(t)    = sum_{s != t} w_s^{T(t)} K(t,s) 2 r^2 / sigma^3   (a_t > 0)
 *   gE(s), gI(s) = sum_{t != s, a_t > 0, T(t) = E resp. I} g_t K(t,s)
 * so that gE, gI are the gradient of L = sum_t g_t u(t) with respect to the
 * dendritic weights w^E, w^I.  orc_attraction_grad sums over the near-field
 * leaf pairs of the last orc_attraction (whose tree may have been built with
 * other counts: the counts only chose the pairs); it returns -1 when the
 * attraction has not run or translated pairs are present.  orc_direct_grad
 * sums over all pairs.  Any output may be NULL; g may be NULL (no gE, gI). */
int orc_attraction_grad(const orc_ctx *c, const uint8_t *type, const uint8_t *vac_axon,
                        const uint8_t *vac_dend_e, const uint8_t *vac_dend_i,
                        const double *g, double *u, double *dudsig, double *gE, double *gI);
void orc_direct_grad(int64_t n, const float *x, const float *y, const float *z,
                     const uint8_t *type, const uint8_t *vac_axon, const uint8_t *vac_dend_e,
                     const uint8_t *vac_dend_i, double sigma, const double *g, double *u,
                     double *dudsig, double *gE, double *gI);

/* Expected mean synapse length and its gradient (the loss of the
 * differentiation workload).  An axonal element of t draws dendrite s with
 * probability w_s K(t,s) / u(t) (Eq. 1, Eq. 8; w = the continuous dendritic
 * weights of t's channel, K = exp(-r^2/sigma^2)), so its synapse is
 * l(t) = v(t) / u(t) long on average, with u = sum_s w_s K, v = sum_s w_s K r.
 *   m    = sum_t a_t l(t) / sum_t a_t     (t with a_t > 0 and u(t) > 0)
 *   loss = (m - target)^2
 * out4 = {loss, m, dloss/dsigma, dm/dsigma}; gE, gI (may be NULL: no weight
 * gradient) = dloss/dw^E, dloss/dw^I.  orc_length_loss sums over the
 * near-field leaf pairs of the last orc_attraction (returns -1 without one or
 * with translated pairs); orc_direct_length_loss over all pairs. */
int orc_length_loss(const orc_ctx *c, const uint8_t *type, const uint8_t *vac_axon,
                    const double *we, const double *wi, double target, double *out4,
                    double *gE, double *gI);
void orc_direct_length_loss(int64_t n, const float *x, const float *y, const float *z,
                            const uint8_t *type, const uint8_t *vac_axon, const double *we,
                            const double *wi, double sigma, double target, double *out4,
                            double *gE, double *gI);

/* Vacancy random walk: v <- clamp(v +- 1, 0, 5) per neuron and channel. */
void orc_vacancy_walk(int64_t n, uint64_t seed, uint64_t step, uint8_t *vac_axon,
                      uint8_t *vac_dend_e, uint8_t *vac_dend_i);

/* Subtract formed synapses from the vacancies (vacant = elements - synapses). */
void orc_commit_synapses(int64_t n_syn, const int32_t *syn_pre, const int32_t *syn_post,
                         const uint8_t *syn_type, uint8_t *vac_axon,
                         uint8_t *vac_dend_e, uint8_t *vac_dend_i);

/* ---- introspection (sizes, then copies) ---- */
int64_t orc_num_nodes(const orc_ctx *c);
int64_t orc_num_pairs(const orc_ctx *c);
int     orc_num_pair_depths(const orc_ctx *c);
int64_t orc_num_elements(const orc_ctx *c);
int     orc_far_level(const orc_ctx *c);
void orc_get_keys(const orc_ctx *c, uint64_t *keys_sorted, int32_t *perm);
void orc_get_nodes(const orc_ctx *c, uint8_t *level, uint64_t *prefix, int32_t *first,
                   int32_t *count, int32_t *parent, int32_t *child_first, uint8_t *nchild);
void orc_get_node_sums(const orc_ctx *c, int32_t *sums4 /* n x {aE,aI,wE,wI} */,
                       double *cent6 /* n x {axon xyz, dendrite xyz} */);
void orc_get_pairs(const orc_ctx *c, int32_t *X, int32_t *Y, uint8_t *kind,
                   int32_t *child_first, double *wE, double *wI, int64_t *depth_start);
void orc_get_expansions(const orc_ctx *c, int64_t node, double *A /* 2 x p^3 */,
                        double *M /* 2 x p^3 */, double *B /* 2 x p^3 */);
void orc_get_stats(const orc_ctx *c, int64_t *stats /* 8 */);

/* ---- building blocks exposed for the pin tests ---- */
/* Hermite functions h_0..h_nmax at x (h_n(x) = (-1)^n d^n/dx^n exp(-x^2)). */
void orc_hermite(int nmax, double x, double *h);
/* Morton key of one position (single precision quantisation). */
uint64_t orc_morton(float x, float y, float z, const float origin[3], float side);
/* Hermite coefficients (Eq. 7) of the weighted points about centre c. */
void orc_p2m(int p, double sigma, int64_t n, const double *pts /* n x 3 */,
             const double *w, const double *c, double *A /* p^3 */);
/* Hermite -> Taylor translation: B = M2L(A; (cA - cD)/sigma). */
void orc_m2l(int p, double sigma, const double *A, const double *cA,
             const double *cD, double *B);
/* Evaluate a Taylor expansion about cA at point t. */
double orc_l2p(int p, double sigma, const double *B, const double *cA, const double *t);
/* Evaluate a Hermite expansion about cD at point t. */
double orc_m2p(int p, double sigma, const double *A, const double *cD, const double *t);
/* Philox4x32-10 block and the derived FP64 uniform. */
void   orc_philox(uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint64_t seed, uint32_t c0, uint32_t c1, uint64_t step);

#ifdef __cplusplus
}
#endif
#endif
