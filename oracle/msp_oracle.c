/*
 * msp_oracle.c -- plain FP64 CPU oracle for the FMM synapse search of
 * arXiv 2301.10570 (Noettgen, Czappa, Wolf).  TEST INFRASTRUCTURE ONLY: it is
 * loaded by the tests, the smoke check and the CPU-baseline leg of the
 * benchmark, never by the product path.  It shares no code with the CUDA
 * library.
 *
 * The code follows the paper's steps in the paper's order and notation:
 *   Section 3.2   octree: recursive subdivision, inner nodes carry the sums of
 *                 vacant elements and their centroids
 *   Eq. 8         the attraction u(t) = sum_j w_j exp(-|t - s_j|^2 / sigma^2)
 *   Eq. 7         Hermite coefficients A_alpha of a source box
 *   Eq. 6         Taylor coefficients B_beta about a target box
 *   Algorithm 1   dual descent over (axon box, dendrite box) pairs
 *   Algorithm 2   candidate attractions, total, uniform draw, upper_bound
 *   Section 4     requests are resolved at the dendrite side
 *   (derivatives) du/dsigma and the transposed transform sum_t g_t K(t,s) of
 *                 Eq. 8, the adjoint of the attraction
 * and these readings of the paper (kernel width,
 * sign of Eq. 6, truncation 0 <= alpha_d < p, centroids as expansion centres
 * (or, with centre_mode 1, the boxes' geometric centres),
 * the Hermite-to-Taylor translation derived from Eq. 6 and Eq. 7, the
 * separation/cutoff rule, the leaf rule of Algorithm 1, resolution order).
 *
 * Nothing here is blocked, fused or reordered beyond those definitions:
 * every sum is the plain loop of its formula.
 */
#include "msp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MORTON_BITS 21
#define TAG_DESCEND 1u
#define TAG_LEAF    2u
#define TAG_ACCEPT  3u
#define TAG_WALK    4u
#define MAXP 8
/* A draw whose total attraction is at or below this counts as having no
 * candidate (no partner is drawn).  Every attraction inside the cutoff radius
 * is many orders of magnitude larger (exp(-cutoff^2) times an integer
 * weight); the threshold only keeps sums of terms far below single precision
 * range from deciding a draw. */
#define ORC_MIN_ATTRACTION 1e-30

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplications,     */
/* with the key bumped by the Weyl constants between rounds.                  */
/* ------------------------------------------------------------------------- */
void orc_philox(uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_draw(uint64_t seed, uint32_t c0, uint32_t c1, uint64_t step,
                        uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, (uint32_t)step, (uint32_t)(step >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox(ctr, key, out);
}

/* U in [0,1): the top 53 bits of the first two output words. */
double orc_uniform(uint64_t seed, uint32_t c0, uint32_t c1, uint64_t step)
{
    uint32_t o[4];
    philox_draw(seed, c0, c1, step, o);
    uint64_t bits = (((uint64_t)o[0] << 32) | o[1]) >> 11;
    return (double)bits * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------- */
/* Hermite functions h_n(x) = (-1)^n d^n/dx^n exp(-x^2) = H_n(x) exp(-x^2),   */
/* the functions of Greengard and Strain that Eq. 6 and Eq. 7 refer to, by    */
/* the three-term recurrence of the physicists' Hermite polynomials.          */
/* ------------------------------------------------------------------------- */
void orc_hermite(int nmax, double x, double *h)
{
    h[0] = exp(-x * x);
    if (nmax >= 1) h[1] = 2.0 * x * h[0];
    for (int n = 1; n < nmax; ++n) h[n + 1] = 2.0 * x * h[n] - 2.0 * n * h[n - 1];
}

static double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

/* ------------------------------------------------------------------------- */
/* Morton key: quantise each coordinate to the 2^21 grid of the domain cube   */
/* in single precision (x - o) * scale, round toward -inf, clamp; interleave  */
/* the bits x-major so that bit 3k+2 / 3k+1 / 3k holds bit k of qx / qy / qz. */
/* ------------------------------------------------------------------------- */
static uint32_t quantise(float v, float o, float scale)
{
    float d = v - o;
    float s = d * scale;
    float f = floorf(s);
    if (!(f >= 0.0f)) return 0u;                      /* also catches NaN */
    if (f >= (float)(1u << MORTON_BITS)) return (1u << MORTON_BITS) - 1u;
    return (uint32_t)f;
}

static float morton_scale(float side)
{
    return (float)((double)(1u << MORTON_BITS) / (double)side);
}

uint64_t orc_morton(float x, float y, float z, const float origin[3], float side)
{
    float scale = morton_scale(side);
    uint32_t q[3] = {quantise(x, origin[0], scale), quantise(y, origin[1], scale),
                     quantise(z, origin[2], scale)};
    uint64_t key = 0;
    for (int k = 0; k < MORTON_BITS; ++k) {
        key |= (uint64_t)((q[0] >> k) & 1u) << (3 * k + 2);
        key |= (uint64_t)((q[1] >> k) & 1u) << (3 * k + 1);
        key |= (uint64_t)((q[2] >> k) & 1u) << (3 * k);
    }
    return key;
}

/* integer box coordinate along dimension d (0=x,1=y,2=z) of a level-l prefix */
static uint32_t prefix_coord(uint64_t prefix, int level, int d)
{
    uint32_t c = 0;
    for (int j = 0; j < level; ++j)
        c |= (uint32_t)((prefix >> (3 * j + (2 - d))) & 1u) << j;
    return c;
}

/* ------------------------------------------------------------------------- */
/* Expansions (Eq. 6, Eq. 7 and their composition)                           */
/* ------------------------------------------------------------------------- */
static int idx3(int p, int a0, int a1, int a2) { return (a0 * p + a1) * p + a2; }

/* A_alpha = 1/alpha! sum_j w_j ((s_j - c)/sigma)^alpha          (Eq. 7) */
void orc_p2m(int p, double sigma, int64_t n, const double *pts, const double *w,
             const double *c, double *A)
{
    for (int i = 0; i < p * p * p; ++i) A[i] = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double y[3];
        for (int d = 0; d < 3; ++d) y[d] = (pts[3 * j + d] - c[d]) / sigma;
        for (int a0 = 0; a0 < p; ++a0)
            for (int a1 = 0; a1 < p; ++a1)
                for (int a2 = 0; a2 < p; ++a2)
                    A[idx3(p, a0, a1, a2)] += w[j] * pow(y[0], a0) * pow(y[1], a1) *
                                              pow(y[2], a2) /
                                              (factorial(a0) * factorial(a1) * factorial(a2));
    }
}

/* Composition of Eq. 7 with the Taylor expansion of Eq. 6: with
 * Delta = (cA - cD)/sigma,
 *   B_beta = (-1)^|beta| / beta!  sum_alpha A_alpha h_{alpha+beta}(Delta)
 * where h_gamma(Delta) = prod_d h_{gamma_d}(Delta_d). */
void orc_m2l(int p, double sigma, const double *A, const double *cA, const double *cD,
             double *B)
{
    double H[3][2 * MAXP];
    for (int d = 0; d < 3; ++d) orc_hermite(2 * p - 2, (cA[d] - cD[d]) / sigma, H[d]);
    for (int b0 = 0; b0 < p; ++b0)
        for (int b1 = 0; b1 < p; ++b1)
            for (int b2 = 0; b2 < p; ++b2) {
                double s = 0.0;
                for (int a0 = 0; a0 < p; ++a0)
                    for (int a1 = 0; a1 < p; ++a1)
                        for (int a2 = 0; a2 < p; ++a2)
                            s += A[idx3(p, a0, a1, a2)] * H[0][a0 + b0] * H[1][a1 + b1] *
                                 H[2][a2 + b2];
                double sign = ((b0 + b1 + b2) & 1) ? -1.0 : 1.0;
                B[idx3(p, b0, b1, b2)] =
                    sign / (factorial(b0) * factorial(b1) * factorial(b2)) * s;
            }
}

/* u(t) ~ sum_beta B_beta ((t - cA)/sigma)^beta                   (Eq. 6) */
double orc_l2p(int p, double sigma, const double *B, const double *cA, const double *t)
{
    double x[3];
    for (int d = 0; d < 3; ++d) x[d] = (t[d] - cA[d]) / sigma;
    double u = 0.0;
    for (int b0 = 0; b0 < p; ++b0)
        for (int b1 = 0; b1 < p; ++b1)
            for (int b2 = 0; b2 < p; ++b2)
                u += B[idx3(p, b0, b1, b2)] * pow(x[0], b0) * pow(x[1], b1) * pow(x[2], b2);
    return u;
}

/* u(t) ~ sum_alpha A_alpha h_alpha((t - cD)/sigma)               (Eq. 7) */
double orc_m2p(int p, double sigma, const double *A, const double *cD, const double *t)
{
    double H[3][MAXP];
    for (int d = 0; d < 3; ++d) orc_hermite(p - 1, (t[d] - cD[d]) / sigma, H[d]);
    double u = 0.0;
    for (int a0 = 0; a0 < p; ++a0)
        for (int a1 = 0; a1 < p; ++a1)
            for (int a2 = 0; a2 < p; ++a2)
                u += A[idx3(p, a0, a1, a2)] * H[0][a0] * H[1][a1] * H[2][a2];
    return u;
}

/* ------------------------------------------------------------------------- */
/* Context                                                                    */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint8_t level;
    uint64_t prefix;
    int32_t first, count, parent, child_first;
    uint8_t nchild;
    int64_t sa[2], sw[2];     /* vacant axons (E,I), vacant dendrites (E,I) */
    double ca[3], cd[3];      /* axon / dendrite centroids                 */
    double gc[3];             /* geometric centre                          */
} node_t;

typedef struct {
    int32_t X, Y;
    uint8_t kind;
    int64_t child_first;
    double w[2];
} pair_t;

typedef struct {
    int32_t X, Y;
    int64_t q;        /* traversal pair id, -1 below a far pair */
    uint8_t nb;       /* a draw on the path was near a CDF boundary */
} item_t;

struct orc_ctx {
    orc_config cfg;
    int64_t n;
    /* sorted (Morton order) data */
    uint64_t *keys;
    int32_t *perm;
    double *pos;              /* n x 3, sorted order */
    uint8_t *type, *va, *vde, *vdi;   /* sorted order */
    /* original-order inputs needed by the selection */
    uint8_t *o_type, *o_va, *o_vde, *o_vdi;
    int64_t *elem_off;        /* exclusive prefix of vac_axon, original order */
    int64_t n_elem;
    /* tree */
    node_t *nodes;
    int64_t n_nodes, cap_nodes;
    int32_t *leaf_of;         /* sorted point -> leaf node */
    int l_far;
    long long *g2;            /* pruning threshold per level */
    /* expansions (all nodes at level >= l_far): [node][channel][p^3] */
    double *A, *M, *B;
    /* traversal */
    pair_t *pairs;
    int64_t n_pairs, cap_pairs;
    int64_t depth_start[128];
    int n_depths;
    int attraction_done;
    int64_t stats[8];
};

orc_ctx *orc_create(const orc_config *cfg)
{
    if (cfg->p < 1 || cfg->p > MAXP || cfg->sigma <= 0.0 || cfg->leaf_capacity < 1 ||
        cfg->max_depth < 0 || cfg->max_depth > MORTON_BITS || !(cfg->side > 0.0f))
        return NULL;
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    c->cfg = *cfg;
    return c;
}

static void free_tree(orc_ctx *c)
{
    free(c->keys); free(c->perm); free(c->pos); free(c->type); free(c->va);
    free(c->vde); free(c->vdi); free(c->o_type); free(c->o_va); free(c->o_vde);
    free(c->o_vdi); free(c->elem_off); free(c->nodes); free(c->leaf_of); free(c->g2);
    free(c->A); free(c->M); free(c->B); free(c->pairs);
    c->keys = NULL; c->perm = NULL; c->pos = NULL; c->type = c->va = c->vde = c->vdi = NULL;
    c->o_type = c->o_va = c->o_vde = c->o_vdi = NULL; c->elem_off = NULL; c->nodes = NULL;
    c->leaf_of = NULL; c->g2 = NULL; c->A = c->M = c->B = NULL; c->pairs = NULL;
    c->n_nodes = c->cap_nodes = c->n_pairs = c->cap_pairs = 0;
    c->attraction_done = 0;
}

void orc_destroy(orc_ctx *c)
{
    if (!c) return;
    free_tree(c);
    free(c);
}

/* ------------------------------------------------------------------------- */
/* a1-a4: keys, sort, octree, aggregates                                      */
/* ------------------------------------------------------------------------- */
typedef struct { uint64_t key; int32_t idx; } keyidx_t;

static int cmp_keyidx(const void *a, const void *b)
{
    const keyidx_t *x = (const keyidx_t *)a, *y = (const keyidx_t *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);     /* stable: original order */
}

static int64_t push_node(orc_ctx *c, node_t nd)
{
    if (c->n_nodes == c->cap_nodes) {
        c->cap_nodes = c->cap_nodes ? 2 * c->cap_nodes : 1024;
        c->nodes = (node_t *)realloc(c->nodes, (size_t)c->cap_nodes * sizeof(node_t));
    }
    c->nodes[c->n_nodes] = nd;
    return c->n_nodes++;
}

int orc_build_tree(orc_ctx *c, int64_t n, const float *x, const float *y, const float *z,
                   const uint8_t *type, const uint8_t *vac_axon, const uint8_t *vac_dend_e,
                   const uint8_t *vac_dend_i)
{
    free_tree(c);
    const orc_config *cfg = &c->cfg;
    c->n = n;
    size_t nn = (size_t)(n > 0 ? n : 1);
    c->keys = (uint64_t *)malloc(nn * sizeof(uint64_t));
    c->perm = (int32_t *)malloc(nn * sizeof(int32_t));
    c->pos = (double *)malloc(3 * nn * sizeof(double));
    c->type = (uint8_t *)malloc(nn); c->va = (uint8_t *)malloc(nn);
    c->vde = (uint8_t *)malloc(nn); c->vdi = (uint8_t *)malloc(nn);
    c->o_type = (uint8_t *)malloc(nn); c->o_va = (uint8_t *)malloc(nn);
    c->o_vde = (uint8_t *)malloc(nn); c->o_vdi = (uint8_t *)malloc(nn);
    c->elem_off = (int64_t *)malloc((nn + 1) * sizeof(int64_t));
    c->leaf_of = (int32_t *)malloc(nn * sizeof(int32_t));

    /* a1: Morton keys;  a2: stable sort by key */
    keyidx_t *ki = (keyidx_t *)malloc(nn * sizeof(keyidx_t));
    for (int64_t i = 0; i < n; ++i) {
        ki[i].key = orc_morton(x[i], y[i], z[i], cfg->origin, cfg->side);
        ki[i].idx = (int32_t)i;
    }
    qsort(ki, (size_t)n, sizeof(keyidx_t), cmp_keyidx);
    for (int64_t i = 0; i < n; ++i) {
        int32_t j = ki[i].idx;
        c->keys[i] = ki[i].key;
        c->perm[i] = j;
        c->pos[3 * i + 0] = x[j];
        c->pos[3 * i + 1] = y[j];
        c->pos[3 * i + 2] = z[j];
        c->type[i] = type[j]; c->va[i] = vac_axon[j];
        c->vde[i] = vac_dend_e[j]; c->vdi[i] = vac_dend_i[j];
    }
    free(ki);
    memcpy(c->o_type, type, (size_t)n); memcpy(c->o_va, vac_axon, (size_t)n);
    memcpy(c->o_vde, vac_dend_e, (size_t)n); memcpy(c->o_vdi, vac_dend_i, (size_t)n);
    c->elem_off[0] = 0;
    for (int64_t i = 0; i < n; ++i) c->elem_off[i + 1] = c->elem_off[i] + vac_axon[i];
    c->n_elem = c->elem_off[n];

    /* a3: breadth-first subdivision.  A node is split while it holds more than
     * leaf_capacity points and lies above max_depth; its non-empty octants
     * become its children, in octant order.  Processing nodes in index order
     * and appending children yields the canonical (level, key) order. */
    node_t root;
    memset(&root, 0, sizeof(root));
    root.count = (int32_t)n;
    root.parent = -1;
    root.child_first = -1;
    push_node(c, root);
    for (int64_t i = 0; i < c->n_nodes; ++i) {
        node_t nd = c->nodes[i];
        if (nd.count <= cfg->leaf_capacity || nd.level >= cfg->max_depth) continue;
        int shift = 3 * (MORTON_BITS - (nd.level + 1));
        int64_t start = nd.first, end = (int64_t)nd.first + nd.count;
        int32_t cf = -1;
        uint8_t nch = 0;
        int64_t s = start;
        while (s < end) {
            uint64_t oct = (c->keys[s] >> shift) & 7u;
            int64_t e = s;
            while (e < end && ((c->keys[e] >> shift) & 7u) == oct) ++e;
            node_t ch;
            memset(&ch, 0, sizeof(ch));
            ch.level = (uint8_t)(nd.level + 1);
            ch.prefix = c->keys[s] >> shift;
            ch.first = (int32_t)s;
            ch.count = (int32_t)(e - s);
            ch.parent = (int32_t)i;
            ch.child_first = -1;
            int64_t id = push_node(c, ch);
            if (cf < 0) cf = (int32_t)id;
            ++nch;
            s = e;
        }
        c->nodes[i].child_first = cf;
        c->nodes[i].nchild = nch;
    }

    /* a4: sums of vacant elements and centroids (Section 3.2; the axon
     * centroid of Section 4).  Channel T of an axon is the neuron's type;
     * both dendrite counts of a neuron enter the dendrite centroid. */
    double side = cfg->side;
    for (int64_t i = 0; i < c->n_nodes; ++i) {
        node_t *nd = &c->nodes[i];
        double swa = 0, swd = 0, pa[3] = {0, 0, 0}, pd[3] = {0, 0, 0};
        for (int64_t s = nd->first; s < (int64_t)nd->first + nd->count; ++s) {
            int t = c->type[s] ? 1 : 0;
            nd->sa[t] += c->va[s];
            nd->sw[0] += c->vde[s];
            nd->sw[1] += c->vdi[s];
            double wa = c->va[s], wd = (double)c->vde[s] + (double)c->vdi[s];
            swa += wa; swd += wd;
            for (int d = 0; d < 3; ++d) {
                pa[d] += wa * c->pos[3 * s + d];
                pd[d] += wd * c->pos[3 * s + d];
            }
        }
        double bs = side / ldexp(1.0, nd->level);
        for (int d = 0; d < 3; ++d) {
            double gc = cfg->origin[d] + (prefix_coord(nd->prefix, nd->level, d) + 0.5) * bs;
            nd->ca[d] = swa > 0 ? pa[d] / swa : gc;
            nd->cd[d] = swd > 0 ? pd[d] / swd : gc;
            nd->gc[d] = gc;
        }
        if (nd->child_first < 0)
            for (int64_t s = nd->first; s < (int64_t)nd->first + nd->count; ++s)
                c->leaf_of[s] = (int32_t)i;
    }

    /* level thresholds: far-field eligibility and pruning gap */
    c->l_far = cfg->max_depth + 1;
    for (int l = 0; l <= cfg->max_depth; ++l)
        if (side / ldexp(1.0, l + 1) <= cfg->rho_max * cfg->sigma) { c->l_far = l; break; }
    if (cfg->mac_mode == 1) c->l_far = 0;   /* Algorithm 2 has no size criterion */
    c->g2 = (long long *)malloc((MORTON_BITS + 1) * sizeof(long long));
    for (int l = 0; l <= MORTON_BITS; ++l) {
        double bl = side / ldexp(1.0, l);
        double r = cfg->cutoff * cfg->sigma / bl;
        c->g2[l] = (long long)ceil(r * r);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* a5: dual traversal (Algorithm 1's pairing rule) with the separation rule   */
/* ------------------------------------------------------------------------- */
static int is_leaf(const node_t *nd) { return nd->child_first < 0; }

static uint8_t classify(const orc_ctx *c, int32_t xi, int32_t yi)
{
    /* Pairs are pruned by the cutoff only.  A pair without vacant axonal or
     * dendritic elements attracts with exactly zero and is never chosen by
     * the descent, so keeping it changes no result; the lists then depend on
     * the positions alone. */
    const node_t *X = &c->nodes[xi], *Y = &c->nodes[yi];
    int lf = X->level > Y->level ? X->level : Y->level;
    long long gsum = 0, gmax = 0;
    for (int d = 0; d < 3; ++d) {
        long long lox = (long long)prefix_coord(X->prefix, X->level, d) << (lf - X->level);
        long long hix = lox + (1ll << (lf - X->level));
        long long loy = (long long)prefix_coord(Y->prefix, Y->level, d) << (lf - Y->level);
        long long hiy = loy + (1ll << (lf - Y->level));
        long long g = 0;
        if (loy - hix > g) g = loy - hix;
        if (lox - hiy > g) g = lox - hiy;
        gsum += g * g;
        if (g > gmax) gmax = g;
    }
    if (gsum >= c->g2[lf]) return ORC_PRUNED;
    if (c->cfg.mac_mode == 1) {
        /* Algorithm 2 (choose_target): a leaf on either side is evaluated
         * directly; an inner dendrite box holding more than c1 vacant
         * dendritic elements is evaluated by an expansion (Hermite when the
         * axon box holds more than c2 vacant axonal elements, else Taylor:
         * here both are the one translation of Eq. 7 by Eq. 6); any other
         * inner pair directly, i.e. refined down to its leaf pairs.  No box
         * is expanded against itself (self pairs stay excluded). */
        if (is_leaf(X) && is_leaf(Y)) return ORC_P2P;
        if (!is_leaf(X) && !is_leaf(Y) && xi != yi && Y->sw[0] + Y->sw[1] > c->cfg.c1)
            return ORC_FAR;
        return ORC_SPLIT;
    }
    int lmin = X->level < Y->level ? X->level : Y->level;
    if (lmin >= c->l_far && gmax >= 1 &&
        (long long)X->count * (long long)Y->count >= c->cfg.m2l_min_pairs)
        return ORC_FAR;
    if (is_leaf(X) && is_leaf(Y)) return ORC_P2P;
    return ORC_SPLIT;
}

static void push_pair(orc_ctx *c, int32_t X, int32_t Y)
{
    if (c->n_pairs == c->cap_pairs) {
        c->cap_pairs = c->cap_pairs ? 2 * c->cap_pairs : 4096;
        c->pairs = (pair_t *)realloc(c->pairs, (size_t)c->cap_pairs * sizeof(pair_t));
    }
    pair_t pr;
    memset(&pr, 0, sizeof(pr));
    pr.X = X; pr.Y = Y; pr.child_first = -1;
    c->pairs[c->n_pairs++] = pr;
}

/* expansion centres of a box: the axon / dendrite centroids, or (centre_mode
 * 1) the geometric centre for both, so that a translation depends only on
 * the boxes' levels and integer offset */
static const double *centre_a(const orc_ctx *c, const node_t *nd)
{
    return c->cfg.centre_mode ? nd->gc : nd->ca;
}

static const double *centre_d(const orc_ctx *c, const node_t *nd)
{
    return c->cfg.centre_mode ? nd->gc : nd->cd;
}

static int64_t expansion_off(const orc_ctx *c, int64_t node, int ch)
{
    int p = c->cfg.p;
    return (node * 2 + ch) * (int64_t)(p * p * p);
}

int orc_attraction(orc_ctx *c, double *u)
{
    const orc_config *cfg = &c->cfg;
    const int p = cfg->p, p3 = p * p * p;
    const double sigma = cfg->sigma;
    int64_t n = c->n;
    memset(c->stats, 0, sizeof(c->stats));

    /* dual traversal, breadth first.  A split pair's children are stored as
     * one contiguous block, X-child major:
     *   both inner:      (X_i, Y_k) for all children i of X, k of Y
     *   X leaf:          (X, Y_k)
     *   Y leaf:          (X_i, Y)                                         */
    c->n_pairs = 0;
    c->n_depths = 0;
    if (n > 0) push_pair(c, 0, 0);
    int64_t start = 0;
    while (start < c->n_pairs) {
        int64_t end = c->n_pairs;
        c->depth_start[c->n_depths++] = start;
        for (int64_t q = start; q < end; ++q) {
            pair_t *pr = &c->pairs[q];
            pr->kind = classify(c, pr->X, pr->Y);
            if (pr->kind != ORC_SPLIT) continue;
            const node_t *X = &c->nodes[pr->X], *Y = &c->nodes[pr->Y];
            int64_t cf = c->n_pairs;
            int32_t X0 = pr->X, Y0 = pr->Y;
            if (!is_leaf(X) && !is_leaf(Y)) {
                for (int i = 0; i < X->nchild; ++i)
                    for (int k = 0; k < Y->nchild; ++k)
                        push_pair(c, X->child_first + i, Y->child_first + k);
            } else if (is_leaf(X)) {
                for (int k = 0; k < Y->nchild; ++k) push_pair(c, X0, Y->child_first + k);
            } else {
                for (int i = 0; i < X->nchild; ++i) push_pair(c, X->child_first + i, Y0);
            }
            c->pairs[q].child_first = cf;
        }
        start = end;
    }
    c->depth_start[c->n_depths] = c->n_pairs;

    /* a6: Hermite coefficients (Eq. 7) of the dendrite weights and axon
     * moments about the box centroids, for every box at level >= l_far */
    free(c->A); free(c->M); free(c->B);
    size_t ecount = (size_t)(c->n_nodes > 0 ? c->n_nodes : 1) * 2 * p3;
    c->A = (double *)calloc(ecount, sizeof(double));
    c->M = (double *)calloc(ecount, sizeof(double));
    c->B = (double *)calloc(ecount, sizeof(double));
    for (int64_t i = 0; i < c->n_nodes; ++i) {
        const node_t *nd = &c->nodes[i];
        if (nd->level < c->l_far) continue;
        for (int64_t s = nd->first; s < (int64_t)nd->first + nd->count; ++s) {
            double yd[3], xa[3];
            for (int d = 0; d < 3; ++d) {
                yd[d] = (c->pos[3 * s + d] - centre_d(c, nd)[d]) / sigma;
                xa[d] = (c->pos[3 * s + d] - centre_a(c, nd)[d]) / sigma;
            }
            int t = c->type[s] ? 1 : 0;
            for (int a0 = 0; a0 < p; ++a0)
                for (int a1 = 0; a1 < p; ++a1)
                    for (int a2 = 0; a2 < p; ++a2) {
                        int id = idx3(p, a0, a1, a2);
                        double fa = factorial(a0) * factorial(a1) * factorial(a2);
                        double ya = pow(yd[0], a0) * pow(yd[1], a1) * pow(yd[2], a2);
                        c->A[expansion_off(c, i, 0) + id] += c->vde[s] * ya / fa;
                        c->A[expansion_off(c, i, 1) + id] += c->vdi[s] * ya / fa;
                        /* M_beta = sum_t a_t x_t^beta, the target-side moment
                         * that turns a Taylor expansion into a box sum */
                        double xb = pow(xa[0], a0) * pow(xa[1], a1) * pow(xa[2], a2);
                        c->M[expansion_off(c, i, t) + id] += c->va[s] * xb;
                    }
        }
    }

    /* a7: M2L for every far pair; accumulates B(X) and the box-pair
     * attraction W(X,Y) = sum_t a_t sum_beta B_beta(X<-Y) x_t^beta */
    double Bp[MAXP * MAXP * MAXP];
    for (int64_t q = 0; q < c->n_pairs; ++q) {
        pair_t *pr = &c->pairs[q];
        if (pr->kind != ORC_FAR) continue;
        c->stats[1]++;
        const node_t *X = &c->nodes[pr->X], *Y = &c->nodes[pr->Y];
        for (int ch = 0; ch < 2; ++ch) {
            orc_m2l(p, sigma, &c->A[expansion_off(c, pr->Y, ch)], centre_a(c, X),
                    centre_d(c, Y), Bp);
            double w = 0.0;
            for (int b = 0; b < p3; ++b) {
                c->B[expansion_off(c, pr->X, ch) + b] += Bp[b];
                w += Bp[b] * c->M[expansion_off(c, pr->X, ch) + b];
            }
            pr->w[ch] = w;
        }
    }

    /* a8 + a9: L2P from every box at level >= l_far that holds the target,
     * then the exact near field (Eq. 8) over the P2P leaf pairs */
    double *uu = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    for (int64_t s = 0; s < n; ++s) {
        if (c->va[s] == 0) continue;
        int t = c->type[s] ? 1 : 0;
        int64_t nd = c->leaf_of[s];
        while (nd >= 0) {
            if (c->nodes[nd].level >= c->l_far)
                uu[s] += orc_l2p(p, sigma, &c->B[expansion_off(c, nd, t)],
                                 centre_a(c, &c->nodes[nd]), &c->pos[3 * s]);
            nd = c->nodes[nd].parent;
        }
    }
    double inv_s2 = 1.0 / (sigma * sigma);
    for (int64_t q = 0; q < c->n_pairs; ++q) {
        pair_t *pr = &c->pairs[q];
        if (pr->kind != ORC_P2P) continue;
        c->stats[2]++;
        const node_t *X = &c->nodes[pr->X], *Y = &c->nodes[pr->Y];
        for (int64_t t = X->first; t < (int64_t)X->first + X->count; ++t) {
            if (c->va[t] == 0) continue;
            int ch = c->type[t] ? 1 : 0;
            double part = 0.0;
            for (int64_t s = Y->first; s < (int64_t)Y->first + Y->count; ++s) {
                if (s == t) continue;
                double d2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    double e = c->pos[3 * t + d] - c->pos[3 * s + d];
                    d2 += e * e;
                }
                double w = ch ? c->vdi[s] : c->vde[s];
                part += w * exp(-d2 * inv_s2);
                c->stats[3]++;
            }
            uu[t] += part;
            pr->w[ch] += c->va[t] * part;
        }
    }
    for (int64_t s = 0; s < n; ++s) u[c->perm[s]] = c->va[s] ? uu[s] : 0.0;
    free(uu);

    /* a10: the attraction of a split pair is the sum over its child block,
     * deepest pairs first */
    for (int d = c->n_depths - 1; d >= 0; --d)
        for (int64_t q = c->depth_start[d]; q < c->depth_start[d + 1]; ++q) {
            pair_t *pr = &c->pairs[q];
            if (pr->kind != ORC_SPLIT) continue;
            const node_t *X = &c->nodes[pr->X], *Y = &c->nodes[pr->Y];
            int64_t nb = (int64_t)(is_leaf(X) ? 1 : X->nchild) * (is_leaf(Y) ? 1 : Y->nchild);
            double w0 = 0.0, w1 = 0.0;
            for (int64_t k = 0; k < nb; ++k) {
                w0 += c->pairs[pr->child_first + k].w[0];
                w1 += c->pairs[pr->child_first + k].w[1];
            }
            pr->w[0] = w0; pr->w[1] = w1;
        }
    c->stats[0] = c->n_pairs;
    c->attraction_done = 1;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* a11: Algorithm 1 / Algorithm 2                                             */
/* ------------------------------------------------------------------------- */

/* W(X, Y) of one channel from the expansions, for pairs below a far pair */
static double far_w(const orc_ctx *c, int32_t X, int32_t Y, int ch)
{
    int p = c->cfg.p, p3 = p * p * p;
    double Bp[MAXP * MAXP * MAXP];
    orc_m2l(p, c->cfg.sigma, &c->A[expansion_off(c, Y, ch)], centre_a(c, &c->nodes[X]),
            centre_d(c, &c->nodes[Y]), Bp);
    double w = 0.0;
    for (int b = 0; b < p3; ++b) w += Bp[b] * c->M[expansion_off(c, X, ch) + b];
    return w;
}

/* Algorithm 2's last three steps: total, uniform draw in [0,total),
 * upper_bound over the inclusive prefix sums.  Negative candidates (possible
 * only through truncation) count as zero.  Returns -1 when the total is at
 * most ORC_MIN_ATTRACTION.
 * *nb is set when r falls within tol*total of an inner boundary. */
static int draw_index(const double *w, int k, double U, double tol, uint8_t *nb)
{
    double pre[64];
    double tot = 0.0;
    for (int i = 0; i < k; ++i) {
        tot += w[i] > 0.0 ? w[i] : 0.0;
        pre[i] = tot;
    }
    if (!(tot > ORC_MIN_ATTRACTION)) return -1;
    double r = U * tot;
    int pick = -1;
    for (int i = 0; i < k; ++i)
        if (pre[i] > r) { pick = i; break; }
    if (pick < 0)
        for (int i = k - 1; i >= 0; --i)
            if (w[i] > 0.0) { pick = i; break; }
    for (int i = 0; i + 1 < k; ++i)
        if (fabs(r - pre[i]) <= tol * tot) *nb = 1;
    return pick;
}

static void push_item(item_t **v, int64_t *n, int64_t *cap, item_t it)
{
    if (*n == *cap) {
        *cap = *cap ? 2 * *cap : 1024;
        *v = (item_t *)realloc(*v, (size_t)*cap * sizeof(item_t));
    }
    (*v)[(*n)++] = it;
}

typedef struct { int32_t s; uint8_t ch; uint32_t prio; int64_t e; } req_t;

static int cmp_req(const void *a, const void *b)
{
    const req_t *x = (const req_t *)a, *y = (const req_t *)b;
    if (x->s != y->s) return x->s < y->s ? -1 : 1;
    if (x->ch != y->ch) return x->ch < y->ch ? -1 : 1;
    if (x->prio != y->prio) return x->prio < y->prio ? -1 : 1;
    return (x->e > y->e) - (x->e < y->e);
}

int64_t orc_select_partners(orc_ctx *c, uint64_t step, int32_t *partner,
                            uint8_t *near_boundary, uint8_t *accepted, int32_t *syn_pre,
                            int32_t *syn_post, uint8_t *syn_type)
{
    if (!c->attraction_done) return -1;
    const orc_config *cfg = &c->cfg;
    const double tol = cfg->boundary_tol;
    const double inv_s2 = 1.0 / (cfg->sigma * cfg->sigma);
    const double rc2 = (cfg->cutoff * cfg->sigma) * (cfg->cutoff * cfg->sigma);
    int64_t n_elem = c->n_elem;
    for (int64_t e = 0; e < n_elem; ++e) { partner[e] = -1; near_boundary[e] = 0; accepted[e] = 0; }
    int64_t draws = 0, bdraws = 0;

    for (int ch = 0; ch < 2; ++ch) {
        item_t *cur = NULL, *nxt = NULL;
        int64_t ncur = 0, ccur = 0, nnxt = 0, cnxt = 0;
        if (c->n > 0 && c->nodes[0].sa[ch] > 0 && c->pairs[0].w[ch] > ORC_MIN_ATTRACTION) {
            item_t it = {0, 0, 0, 0};
            push_item(&cur, &ncur, &ccur, it);
        }
        while (ncur > 0) {
            nnxt = 0;
            for (int64_t ii = 0; ii < ncur; ++ii) {
                item_t it = cur[ii];
                const node_t *X = &c->nodes[it.X], *Y = &c->nodes[it.Y];
                int split = it.q >= 0 && c->pairs[it.q].kind == ORC_SPLIT;
                int64_t cf = split ? c->pairs[it.q].child_first : -1;
                if (is_leaf(X) && is_leaf(Y)) {
                    /* form_synapse: every vacant element of channel ch in X
                     * draws one dendrite neuron of Y, s != t, with weight
                     * w_s K(t, s) (Eq. 8), the kernel truncated at the same
                     * cutoff radius that prunes box pairs */
                    double w[1024];
                    double *wp = Y->count <= 1024 ? w : (double *)malloc(Y->count * sizeof(double));
                    for (int64_t t = X->first; t < (int64_t)X->first + X->count; ++t) {
                        if ((c->type[t] ? 1 : 0) != ch || c->va[t] == 0) continue;
                        double tot = 0.0;
                        for (int64_t s = Y->first; s < (int64_t)Y->first + Y->count; ++s) {
                            double ws = 0.0;
                            if (s != t) {
                                double d2 = 0.0;
                                for (int d = 0; d < 3; ++d) {
                                    double e = c->pos[3 * t + d] - c->pos[3 * s + d];
                                    d2 += e * e;
                                }
                                ws = d2 < rc2 ? (ch ? c->vdi[s] : c->vde[s]) * exp(-d2 * inv_s2) : 0.0;
                            }
                            wp[s - Y->first] = ws;
                            tot += ws;
                        }
                        int32_t to = c->perm[t];
                        for (int k = 0; k < c->va[t]; ++k) {
                            int64_t e = c->elem_off[to] + k;
                            near_boundary[e] = it.nb;
                            if (!(tot > ORC_MIN_ATTRACTION)) continue;
                            double U = orc_uniform(cfg->seed, (uint32_t)to,
                                                   (uint32_t)k | ((uint32_t)ch << 8) | (TAG_LEAF << 16),
                                                   step);
                            uint8_t nb = 0;
                            /* inverse CDF over the (up to Y->count) sources */
                            double r = U * tot, pre = 0.0;
                            int64_t pick = -1;
                            for (int64_t s = 0; s < Y->count; ++s) {
                                pre += wp[s];
                                if (pick < 0 && pre > r) pick = s;
                                if (s + 1 < Y->count && fabs(r - pre) <= tol * tot) nb = 1;
                            }
                            if (pick < 0)
                                for (int64_t s = Y->count - 1; s >= 0; --s)
                                    if (wp[s] > 0.0) { pick = s; break; }
                            partner[e] = c->perm[Y->first + pick];
                            near_boundary[e] = (uint8_t)(it.nb | nb);
                            draws++; bdraws += nb;
                        }
                    }
                    if (wp != w) free(wp);
                } else if (is_leaf(X)) {
                    /* choose_target for the whole axon leaf */
                    double w[8];
                    for (int k = 0; k < Y->nchild; ++k)
                        w[k] = split ? c->pairs[cf + k].w[ch] : far_w(c, it.X, Y->child_first + k, ch);
                    double U = orc_uniform(cfg->seed, (uint32_t)it.X,
                                           (uint32_t)(Y->level + 1) | ((uint32_t)ch << 8) |
                                               (TAG_DESCEND << 16),
                                           step);
                    uint8_t nb = 0;
                    int k = draw_index(w, Y->nchild, U, tol, &nb);
                    draws++; bdraws += nb;
                    if (k >= 0) {
                        item_t nx = {it.X, Y->child_first + k, split ? cf + k : -1,
                                     (uint8_t)(it.nb | nb)};
                        push_item(&nxt, &nnxt, &cnxt, nx);
                    }
                } else if (is_leaf(Y)) {
                    /* the dendrite side is a leaf: each axon child with vacant
                     * elements keeps the leaf without a draw */
                    for (int i = 0; i < X->nchild; ++i) {
                        int32_t xc = X->child_first + i;
                        if (c->nodes[xc].sa[ch] == 0) continue;
                        if (split && !(c->pairs[cf + i].w[ch] > ORC_MIN_ATTRACTION)) continue;
                        item_t nx = {xc, it.Y, split ? cf + i : -1, it.nb};
                        push_item(&nxt, &nnxt, &cnxt, nx);
                    }
                } else {
                    /* both inner: every axon child chooses among the dendrite
                     * children (Algorithm 1, last branch) */
                    for (int i = 0; i < X->nchild; ++i) {
                        int32_t xc = X->child_first + i;
                        if (c->nodes[xc].sa[ch] == 0) continue;
                        double w[8];
                        for (int k = 0; k < Y->nchild; ++k)
                            w[k] = split ? c->pairs[cf + (int64_t)i * Y->nchild + k].w[ch]
                                         : far_w(c, xc, Y->child_first + k, ch);
                        double U = orc_uniform(cfg->seed, (uint32_t)xc,
                                               (uint32_t)(Y->level + 1) | ((uint32_t)ch << 8) |
                                                   (TAG_DESCEND << 16),
                                               step);
                        uint8_t nb = 0;
                        int k = draw_index(w, Y->nchild, U, tol, &nb);
                        draws++; bdraws += nb;
                        if (k >= 0) {
                            item_t nx = {xc, Y->child_first + k,
                                         split ? cf + (int64_t)i * Y->nchild + k : -1,
                                         (uint8_t)(it.nb | nb)};
                            push_item(&nxt, &nnxt, &cnxt, nx);
                        }
                    }
                }
            }
            item_t *tmp = cur; cur = nxt; nxt = tmp;
            int64_t tc = ccur; ccur = cnxt; cnxt = tc;
            ncur = nnxt;
        }
        free(cur); free(nxt);
    }
    c->stats[4] = draws;
    c->stats[5] = bdraws;

    /* a12: requests go to the dendrite neuron; it accepts, per channel, as
     * many as it has vacant dendritic elements, lowest priority first */
    req_t *rq = (req_t *)malloc((size_t)(n_elem > 0 ? n_elem : 1) * sizeof(req_t));
    int64_t nr = 0;
    for (int64_t i = 0; i < c->n; ++i)
        for (int k = 0; k < c->o_va[i]; ++k) {
            int64_t e = c->elem_off[i] + k;
            if (partner[e] < 0) continue;
            uint32_t o[4];
            philox_draw(cfg->seed, (uint32_t)i, (uint32_t)k | (TAG_ACCEPT << 16), step, o);
            req_t r = {partner[e], (uint8_t)(c->o_type[i] ? 1 : 0), o[0], e};
            rq[nr++] = r;
        }
    qsort(rq, (size_t)nr, sizeof(req_t), cmp_req);
    for (int64_t a = 0; a < nr;) {
        int64_t b = a;
        while (b < nr && rq[b].s == rq[a].s && rq[b].ch == rq[a].ch) ++b;
        int cap = rq[a].ch ? c->o_vdi[rq[a].s] : c->o_vde[rq[a].s];
        for (int64_t j = a; j < b && j - a < cap; ++j) accepted[rq[j].e] = 1;
        a = b;
    }
    free(rq);
    int64_t n_syn = 0;
    for (int64_t i = 0; i < c->n; ++i)
        for (int k = 0; k < c->o_va[i]; ++k) {
            int64_t e = c->elem_off[i] + k;
            if (!accepted[e]) continue;
            syn_pre[n_syn] = (int32_t)i;
            syn_post[n_syn] = partner[e];
            syn_type[n_syn] = (uint8_t)(c->o_type[i] ? 1 : 0);
            ++n_syn;
        }
    c->stats[6] = nr;
    c->stats[7] = n_syn;
    return n_syn;
}

/* ------------------------------------------------------------------------- */
/* Eq. 8 by brute force                                                       */
/* ------------------------------------------------------------------------- */
void orc_direct(int64_t n, const float *x, const float *y, const float *z, const uint8_t *type,
                const uint8_t *vac_axon, const uint8_t *vac_dend_e, const uint8_t *vac_dend_i,
                double sigma, int64_t n_targets, const int64_t *targets, double *u)
{
    double inv_s2 = 1.0 / (sigma * sigma);
    for (int64_t k = 0; k < n_targets; ++k) {
        int64_t t = targets[k];
        if (vac_axon[t] == 0) { u[k] = 0.0; continue; }
        const uint8_t *w = type[t] ? vac_dend_i : vac_dend_e;
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == t) continue;
            double dx = (double)x[t] - x[j], dy = (double)y[t] - y[j], dz = (double)z[t] - z[j];
            s += w[j] * exp(-(dx * dx + dy * dy + dz * dz) * inv_s2);
        }
        u[k] = s;
    }
}

/* ------------------------------------------------------------------------- */
/* derivatives of the attraction (Eq. 8)                                      */
/* ------------------------------------------------------------------------- */

/* one (target t, source s) term of every output; t, s caller indices */
static void grad_term(int64_t t, int64_t s, double d2, double sigma, const uint8_t *type,
                      const uint8_t *va, const uint8_t *vde, const uint8_t *vdi,
                      const double *g, double *u, double *dudsig, double *gE, double *gI)
{
    if (va[t] == 0) return;
    double K = exp(-d2 / (sigma * sigma));
    double w = type[t] ? vdi[s] : vde[s];
    if (u) u[t] += w * K;
    if (dudsig) dudsig[t] += w * K * 2.0 * d2 / (sigma * sigma * sigma);
    if (g) {
        double *gs = type[t] ? gI : gE;
        if (gs) gs[s] += g[t] * K;
    }
}

static void zero_outputs(int64_t n, double *u, double *dudsig, double *gE, double *gI)
{
    for (int64_t i = 0; i < n; ++i) {
        if (u) u[i] = 0.0;
        if (dudsig) dudsig[i] = 0.0;
        if (gE) gE[i] = 0.0;
        if (gI) gI[i] = 0.0;
    }
}

int orc_attraction_grad(const orc_ctx *c, const uint8_t *type, const uint8_t *vac_axon,
                        const uint8_t *vac_dend_e, const uint8_t *vac_dend_i,
                        const double *g, double *u, double *dudsig, double *gE, double *gI)
{
    if (!c->attraction_done) return -1;
    for (int64_t q = 0; q < c->n_pairs; ++q)
        if (c->pairs[q].kind == ORC_FAR) return -1;
    zero_outputs(c->n, u, dudsig, gE, gI);
    double sigma = c->cfg.sigma;
    for (int64_t q = 0; q < c->n_pairs; ++q) {
        const pair_t *pr = &c->pairs[q];
        if (pr->kind != ORC_P2P) continue;
        const node_t *X = &c->nodes[pr->X], *Y = &c->nodes[pr->Y];
        for (int64_t t = X->first; t < (int64_t)X->first + X->count; ++t)
            for (int64_t s = Y->first; s < (int64_t)Y->first + Y->count; ++s) {
                if (s == t) continue;
                double d2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    double e = c->pos[3 * t + d] - c->pos[3 * s + d];
                    d2 += e * e;
                }
                grad_term(c->perm[t], c->perm[s], d2, sigma, type, vac_axon, vac_dend_e,
                          vac_dend_i, g, u, dudsig, gE, gI);
            }
    }
    return 0;
}

void orc_direct_grad(int64_t n, const float *x, const float *y, const float *z,
                     const uint8_t *type, const uint8_t *vac_axon, const uint8_t *vac_dend_e,
                     const uint8_t *vac_dend_i, double sigma, const double *g, double *u,
                     double *dudsig, double *gE, double *gI)
{
    zero_outputs(n, u, dudsig, gE, gI);
    for (int64_t t = 0; t < n; ++t)
        for (int64_t s = 0; s < n; ++s) {
            if (s == t) continue;
            double dx = (double)x[t] - x[s], dy = (double)y[t] - y[s], dz = (double)z[t] - z[s];
            grad_term(t, s, dx * dx + dy * dy + dz * dz, sigma, type, vac_axon, vac_dend_e,
                      vac_dend_i, g, u, dudsig, gE, gI);
        }
}

/* ------------------------------------------------------------------------- */
/* expected mean synapse length (Eq. 1 / Eq. 8 probabilities) and its         */
/* derivatives: the loss of the differentiation workload                      */
/* ------------------------------------------------------------------------- */

/* forward terms of one (target t, source s) pair, caller indices: the sums
 * u(t) = sum w K, v(t) = sum w K r and their sigma derivatives */
static void len_fwd_term(int64_t t, int64_t s, double d2, double sigma, const uint8_t *type,
                         const uint8_t *va, const double *we, const double *wi, double *U,
                         double *V, double *dU, double *dV)
{
    if (va[t] == 0) return;
    double K = exp(-d2 / (sigma * sigma));
    double r = sqrt(d2);
    double w = type[t] ? wi[s] : we[s];
    double dK = K * 2.0 * d2 / (sigma * sigma * sigma);    /* dK/dsigma */
    U[t] += w * K;
    V[t] += w * K * r;
    dU[t] += w * dK;
    dV[t] += w * dK * r;
}

/* adjoint terms: dm/dw^T(t)_s += alpha_t K r - beta_t K */
static void len_adj_term(int64_t t, int64_t s, double d2, double sigma, const uint8_t *type,
                         const double *alpha, const double *beta, double *gE, double *gI)
{
    if (alpha[t] == 0.0 && beta[t] == 0.0) return;
    double K = exp(-d2 / (sigma * sigma));
    double *gs = type[t] ? gI : gE;
    gs[s] += alpha[t] * K * sqrt(d2) - beta[t] * K;
}

/* The mean over the targets from their sums, the loss and the sigma
 * derivative; alpha, beta receive the adjoint's per-target coefficients of
 * dloss/dw (already times 2 (m - target)). */
static void len_finish(int64_t n, const uint8_t *va, const double *U, const double *V,
                       const double *dU, const double *dV, double target, double *out4,
                       double *alpha, double *beta)
{
    double A = 0.0, S = 0.0, dS = 0.0;
    for (int64_t t = 0; t < n; ++t) {
        if (va[t] == 0 || !(U[t] > 0.0)) continue;
        A += va[t];
        S += va[t] * V[t] / U[t];
        dS += va[t] * (dV[t] * U[t] - V[t] * dU[t]) / (U[t] * U[t]);
    }
    double m = A > 0.0 ? S / A : 0.0;
    double dm = A > 0.0 ? dS / A : 0.0;
    double f = 2.0 * (m - target);
    out4[0] = (m - target) * (m - target);
    out4[1] = m;
    out4[2] = f * dm;
    out4[3] = dm;
    for (int64_t t = 0; t < n; ++t) {
        alpha[t] = beta[t] = 0.0;
        if (va[t] == 0 || !(U[t] > 0.0) || !(A > 0.0)) continue;
        alpha[t] = f * va[t] / (A * U[t]);
        beta[t] = f * va[t] * V[t] / (A * U[t] * U[t]);
    }
}

/* d2 of a sorted-order point pair of the context */
static double ctx_d2(const orc_ctx *c, int64_t t, int64_t s)
{
    double d2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        double e = c->pos[3 * t + d] - c->pos[3 * s + d];
        d2 += e * e;
    }
    return d2;
}

int orc_length_loss(const orc_ctx *c, const uint8_t *type, const uint8_t *vac_axon,
                    const double *we, const double *wi, double target, double *out4,
                    double *gE, double *gI)
{
    if (!c->attraction_done) return -1;
    for (int64_t q = 0; q < c->n_pairs; ++q)
        if (c->pairs[q].kind == ORC_FAR) return -1;
    int64_t n = c->n;
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *U = (double *)calloc(nn, sizeof(double)), *V = (double *)calloc(nn, sizeof(double));
    double *dU = (double *)calloc(nn, sizeof(double)), *dV = (double *)calloc(nn, sizeof(double));
    double *al = (double *)calloc(nn, sizeof(double)), *be = (double *)calloc(nn, sizeof(double));
    double sigma = c->cfg.sigma;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            len_finish(n, vac_axon, U, V, dU, dV, target, out4, al, be);
            if (!gE || !gI) break;
            for (int64_t i = 0; i < n; ++i) gE[i] = gI[i] = 0.0;
        }
        for (int64_t q = 0; q < c->n_pairs; ++q) {
            const pair_t *pr = &c->pairs[q];
            if (pr->kind != ORC_P2P) continue;
            const node_t *X = &c->nodes[pr->X], *Y = &c->nodes[pr->Y];
            for (int64_t t = X->first; t < (int64_t)X->first + X->count; ++t)
                for (int64_t s = Y->first; s < (int64_t)Y->first + Y->count; ++s) {
                    if (s == t) continue;
                    double d2 = ctx_d2(c, t, s);
                    if (pass == 0)
                        len_fwd_term(c->perm[t], c->perm[s], d2, sigma, type, vac_axon, we, wi,
                                     U, V, dU, dV);
                    else
                        len_adj_term(c->perm[t], c->perm[s], d2, sigma, type, al, be, gE, gI);
                }
        }
    }
    free(U); free(V); free(dU); free(dV); free(al); free(be);
    return 0;
}

void orc_direct_length_loss(int64_t n, const float *x, const float *y, const float *z,
                            const uint8_t *type, const uint8_t *vac_axon, const double *we,
                            const double *wi, double sigma, double target, double *out4,
                            double *gE, double *gI)
{
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *U = (double *)calloc(nn, sizeof(double)), *V = (double *)calloc(nn, sizeof(double));
    double *dU = (double *)calloc(nn, sizeof(double)), *dV = (double *)calloc(nn, sizeof(double));
    double *al = (double *)calloc(nn, sizeof(double)), *be = (double *)calloc(nn, sizeof(double));
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            len_finish(n, vac_axon, U, V, dU, dV, target, out4, al, be);
            if (!gE || !gI) break;
            for (int64_t i = 0; i < n; ++i) gE[i] = gI[i] = 0.0;
        }
        for (int64_t t = 0; t < n; ++t)
            for (int64_t s = 0; s < n; ++s) {
                if (s == t) continue;
                double dx = (double)x[t] - x[s], dy = (double)y[t] - y[s], dz = (double)z[t] - z[s];
                double d2 = dx * dx + dy * dy + dz * dz;
                if (pass == 0)
                    len_fwd_term(t, s, d2, sigma, type, vac_axon, we, wi, U, V, dU, dV);
                else
                    len_adj_term(t, s, d2, sigma, type, al, be, gE, gI);
            }
    }
    free(U); free(V); free(dU); free(dV); free(al); free(be);
}

/* ------------------------------------------------------------------------- */
/* vacancy updates                                                            */
/* ------------------------------------------------------------------------- */
void orc_vacancy_walk(int64_t n, uint64_t seed, uint64_t step, uint8_t *vac_axon,
                      uint8_t *vac_dend_e, uint8_t *vac_dend_i)
{
    uint8_t *v[3] = {vac_axon, vac_dend_e, vac_dend_i};
    for (int64_t i = 0; i < n; ++i)
        for (int ch = 0; ch < 3; ++ch) {
            uint32_t o[4];
            philox_draw(seed, (uint32_t)i, (uint32_t)ch | (TAG_WALK << 16), step, o);
            int nv = (int)v[ch][i] + ((o[0] & 1u) ? 1 : -1);
            if (nv < 0) nv = 0;
            if (nv > 5) nv = 5;
            v[ch][i] = (uint8_t)nv;
        }
}

void orc_commit_synapses(int64_t n_syn, const int32_t *syn_pre, const int32_t *syn_post,
                         const uint8_t *syn_type, uint8_t *vac_axon, uint8_t *vac_dend_e,
                         uint8_t *vac_dend_i)
{
    for (int64_t k = 0; k < n_syn; ++k) {
        if (vac_axon[syn_pre[k]] > 0) vac_axon[syn_pre[k]]--;
        uint8_t *d = syn_type[k] ? vac_dend_i : vac_dend_e;
        if (d[syn_post[k]] > 0) d[syn_post[k]]--;
    }
}

/* ------------------------------------------------------------------------- */
/* introspection                                                              */
/* ------------------------------------------------------------------------- */
int64_t orc_num_nodes(const orc_ctx *c) { return c->n_nodes; }
int64_t orc_num_pairs(const orc_ctx *c) { return c->n_pairs; }
int orc_num_pair_depths(const orc_ctx *c) { return c->n_depths; }
int64_t orc_num_elements(const orc_ctx *c) { return c->n_elem; }
int orc_far_level(const orc_ctx *c) { return c->l_far; }

void orc_get_keys(const orc_ctx *c, uint64_t *keys_sorted, int32_t *perm)
{
    memcpy(keys_sorted, c->keys, (size_t)c->n * sizeof(uint64_t));
    memcpy(perm, c->perm, (size_t)c->n * sizeof(int32_t));
}

void orc_get_nodes(const orc_ctx *c, uint8_t *level, uint64_t *prefix, int32_t *first,
                   int32_t *count, int32_t *parent, int32_t *child_first, uint8_t *nchild)
{
    for (int64_t i = 0; i < c->n_nodes; ++i) {
        level[i] = c->nodes[i].level; prefix[i] = c->nodes[i].prefix;
        first[i] = c->nodes[i].first; count[i] = c->nodes[i].count;
        parent[i] = c->nodes[i].parent; child_first[i] = c->nodes[i].child_first;
        nchild[i] = c->nodes[i].nchild;
    }
}

void orc_get_node_sums(const orc_ctx *c, int32_t *sums4, double *cent6)
{
    for (int64_t i = 0; i < c->n_nodes; ++i) {
        const node_t *nd = &c->nodes[i];
        sums4[4 * i + 0] = (int32_t)nd->sa[0]; sums4[4 * i + 1] = (int32_t)nd->sa[1];
        sums4[4 * i + 2] = (int32_t)nd->sw[0]; sums4[4 * i + 3] = (int32_t)nd->sw[1];
        for (int d = 0; d < 3; ++d) { cent6[6 * i + d] = nd->ca[d]; cent6[6 * i + 3 + d] = nd->cd[d]; }
    }
}

void orc_get_pairs(const orc_ctx *c, int32_t *X, int32_t *Y, uint8_t *kind, int32_t *child_first,
                   double *wE, double *wI, int64_t *depth_start)
{
    for (int64_t q = 0; q < c->n_pairs; ++q) {
        X[q] = c->pairs[q].X; Y[q] = c->pairs[q].Y; kind[q] = c->pairs[q].kind;
        child_first[q] = (int32_t)c->pairs[q].child_first;
        wE[q] = c->pairs[q].w[0]; wI[q] = c->pairs[q].w[1];
    }
    for (int d = 0; d <= c->n_depths; ++d) depth_start[d] = c->depth_start[d];
}

void orc_get_expansions(const orc_ctx *c, int64_t node, double *A, double *M, double *B)
{
    int p3 = c->cfg.p * c->cfg.p * c->cfg.p;
    memcpy(A, &c->A[expansion_off(c, node, 0)], 2 * p3 * sizeof(double));
    memcpy(M, &c->M[expansion_off(c, node, 0)], 2 * p3 * sizeof(double));
    memcpy(B, &c->B[expansion_off(c, node, 0)], 2 * p3 * sizeof(double));
}

void orc_get_stats(const orc_ctx *c, int64_t *stats) { memcpy(stats, c->stats, sizeof(c->stats)); }
