/* msp_neuron.c -- oracle of the Model of Structural Plasticity's neuron side
 * (Section 3.1, Table 1).  TEST INFRASTRUCTURE ONLY.
 *
 * Readings of Section 3.1 taken here (the paper states the model in words):
 *   activity   x <- x + (x0 - x)/tau_x + I + c_in * (number of edges s -> t
 *              whose s spiked in the previous step), then a uniform draw
 *              U in [0,1): the neuron spikes when U < x, unless it spiked in
 *              one of the last `refractory` steps;
 *   calcium    Ca <- Ca - decay * Ca, plus beta on a spike (beta = 5e-4 of
 *              Table 1; the text says 1e-3);
 *   elements   z <- max(z + g(Ca), 0) with the Gaussian growth curve of the
 *              cited model, g(Ca) = mu (2 exp(-((Ca - xi)/zeta)^2) - 1),
 *              xi = (eta + eps)/2, zeta = (eps - eta)/(2 sqrt(ln 2)), so g = 0
 *              at Ca = eta and Ca = eps and g = mu at xi; the axon curve uses
 *              eta_axon, both dendrite curves eta_dend, the calcium after this
 *              step's spike;
 *   deletion   a side with more bound synapses than floor(z) deletes the
 *              excess, uniformly at random; an edge chosen by either side
 *              goes; vacant = floor(z) - bound.
 * Every floating-point operation is single precision, in the order written.
 */
#include "msp_neuron.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "msp_oracle.h"

#define TAG_SPIKE    5u
#define TAG_DEL_AXON 6u
#define TAG_DEL_DEND 7u

static uint32_t draw32(uint64_t seed, uint32_t c0, uint32_t c1, uint64_t step)
{
    uint32_t ctr[4] = {c0, c1, (uint32_t)step, (uint32_t)(step >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox(ctr, key, out);
    return out[0];
}

static float pow2i(int n)   /* 2^n for -126 <= n <= 127 */
{
    uint32_t b = (uint32_t)(n + 127) << 23;
    float f;
    memcpy(&f, &b, sizeof f);
    return f;
}

float orc_expf(float x)
{
    if (x < -87.0f) return 0.0f;
    /* n = nearest integer to x / ln 2 */
    float t = x * 1.44269504f;
    float n = floorf(t + 0.5f);
    /* r = x - n ln 2 with ln 2 = 0.693359375 - 2.12194440e-4 (the first part
     * has few bits, so n times it is exact) */
    float r = x - n * 0.693359375f;
    r = r + n * 2.12194440e-4f;
    /* e^r = sum_{k<=7} r^k / k! (|r| <= 0.35: the next term is below 5e-9) */
    float p = 1.98412698e-4f;
    p = p * r + 1.38888889e-3f;
    p = p * r + 8.33333333e-3f;
    p = p * r + 4.16666667e-2f;
    p = p * r + 1.66666667e-1f;
    p = p * r + 0.5f;
    p = p * r + 1.0f;
    p = p * r + 1.0f;
    return p * pow2i((int)n);
}

float orc_growth(float ca, float eta, float eps, float mu)
{
    float xi = (eta + eps) * 0.5f;
    float zeta = (eps - eta) / (2.0f * 0.832554611f);   /* 2 sqrt(ln 2) */
    float q = (ca - xi) / zeta;
    float e = orc_expf(-(q * q));
    return mu * ((e + e) - 1.0f);
}

void orc_neuron_steps(int64_t n, uint64_t seed, uint64_t first_step, int n_steps,
                      const orc_neuron_params *mp, int64_t n_edges, const int32_t *edge_pre,
                      const int32_t *edge_post, float *x, uint8_t *refractory, float *calcium,
                      float *z_axon, float *z_dend_e, float *z_dend_i, uint8_t *spiked)
{
    int32_t *inp = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    for (int k = 0; k < n_steps; ++k) {
        uint64_t step = first_step + (uint64_t)k;
        memset(inp, 0, (size_t)n * sizeof(int32_t));
        for (int64_t e = 0; e < n_edges; ++e)
            if (spiked[edge_pre[e]]) inp[edge_post[e]] += 1;
        for (int64_t t = 0; t < n; ++t) {
            float xt = x[t];
            float d = mp->x0 - xt;
            d = d / mp->tau_x;
            xt = xt + d;
            xt = xt + mp->background;
            xt = xt + mp->input_per_spike * (float)inp[t];
            x[t] = xt;
            int s = 0;
            if (refractory[t] > 0) {
                refractory[t] -= 1;
            } else {
                uint32_t o = draw32(seed, (uint32_t)t, TAG_SPIKE << 16, step);
                float u = (float)(o >> 8) * (1.0f / 16777216.0f);
                s = u < xt;
                if (s) refractory[t] = (uint8_t)mp->refractory;
            }
            float ca = calcium[t];
            ca = ca - ca * mp->decay_ca;
            if (s) ca = ca + mp->beta_ca;
            calcium[t] = ca;
            float za = z_axon[t] + orc_growth(ca, mp->eta_axon, mp->eps, mp->mu);
            float gd = orc_growth(ca, mp->eta_dend, mp->eps, mp->mu);
            float ze = z_dend_e[t] + gd;
            float zi = z_dend_i[t] + gd;
            z_axon[t] = za > 0.0f ? za : 0.0f;
            z_dend_e[t] = ze > 0.0f ? ze : 0.0f;
            z_dend_i[t] = zi > 0.0f ? zi : 0.0f;
            spiked[t] = (uint8_t)s;
        }
    }
    free(inp);
}

/* deletion order: (group, priority, edge position) */
typedef struct {
    int64_t group;
    uint32_t prio;
    int64_t e;
} del_key;

static int del_cmp(const void *a, const void *b)
{
    const del_key *p = (const del_key *)a, *q = (const del_key *)b;
    if (p->group != q->group) return p->group < q->group ? -1 : 1;
    if (p->prio != q->prio) return p->prio < q->prio ? -1 : 1;
    return p->e < q->e ? -1 : (p->e > q->e);
}

/* marks, per group, the excess[group] edges that come first in the order */
static void choose(int64_t n_edges, del_key *k, const int64_t *excess, uint8_t *del)
{
    qsort(k, (size_t)n_edges, sizeof(del_key), del_cmp);
    int64_t i = 0;
    while (i < n_edges) {
        int64_t j = i;
        while (j < n_edges && k[j].group == k[i].group) ++j;
        int64_t take = excess[k[i].group];
        for (int64_t r = i; r < j && r - i < take; ++r) del[k[r].e] = 1;
        i = j;
    }
}

static int64_t floor_count(float z) { return (int64_t)floorf(z); }

int64_t orc_update_synapses(int64_t n, uint64_t seed, uint64_t step, const float *z_axon,
                            const float *z_dend_e, const float *z_dend_i, int64_t n_edges,
                            int32_t *edge_pre, int32_t *edge_post, uint8_t *edge_type,
                            uint8_t *vac_axon, uint8_t *vac_dend_e, uint8_t *vac_dend_i)
{
    size_t nn = (size_t)(n > 0 ? n : 1), ne = (size_t)(n_edges > 0 ? n_edges : 1);
    int64_t *bound_out = (int64_t *)calloc(nn, sizeof(int64_t));
    int64_t *bound_in = (int64_t *)calloc(2 * nn, sizeof(int64_t));   /* post*2 + type */
    int64_t *ex_out = (int64_t *)calloc(nn, sizeof(int64_t));
    int64_t *ex_in = (int64_t *)calloc(2 * nn, sizeof(int64_t));
    uint8_t *del = (uint8_t *)calloc(ne, 1);
    del_key *k = (del_key *)malloc(ne * sizeof(del_key));
    for (int64_t e = 0; e < n_edges; ++e) {
        bound_out[edge_pre[e]] += 1;
        bound_in[2 * (int64_t)edge_post[e] + edge_type[e]] += 1;
    }
    for (int64_t t = 0; t < n; ++t) {
        int64_t a = bound_out[t] - floor_count(z_axon[t]);
        int64_t de = bound_in[2 * t] - floor_count(z_dend_e[t]);
        int64_t di = bound_in[2 * t + 1] - floor_count(z_dend_i[t]);
        ex_out[t] = a > 0 ? a : 0;
        ex_in[2 * t] = de > 0 ? de : 0;
        ex_in[2 * t + 1] = di > 0 ? di : 0;
    }
    /* the axon side: outgoing edges of each neuron */
    for (int64_t e = 0; e < n_edges; ++e) {
        k[e].group = edge_pre[e];
        k[e].prio = draw32(seed, (uint32_t)e, TAG_DEL_AXON << 16, step);
        k[e].e = e;
    }
    choose(n_edges, k, ex_out, del);
    /* the dendrite side: incoming edges of each neuron and type */
    for (int64_t e = 0; e < n_edges; ++e) {
        k[e].group = 2 * (int64_t)edge_post[e] + edge_type[e];
        k[e].prio = draw32(seed, (uint32_t)e, TAG_DEL_DEND << 16, step);
        k[e].e = e;
    }
    choose(n_edges, k, ex_in, del);
    /* compaction, order kept */
    int64_t m = 0;
    for (int64_t e = 0; e < n_edges; ++e) {
        if (del[e]) continue;
        edge_pre[m] = edge_pre[e];
        edge_post[m] = edge_post[e];
        edge_type[m] = edge_type[e];
        ++m;
    }
    memset(bound_out, 0, nn * sizeof(int64_t));
    memset(bound_in, 0, 2 * nn * sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e) {
        bound_out[edge_pre[e]] += 1;
        bound_in[2 * (int64_t)edge_post[e] + edge_type[e]] += 1;
    }
    for (int64_t t = 0; t < n; ++t) {
        int64_t v[3] = {floor_count(z_axon[t]) - bound_out[t],
                        floor_count(z_dend_e[t]) - bound_in[2 * t],
                        floor_count(z_dend_i[t]) - bound_in[2 * t + 1]};
        uint8_t *dst[3] = {vac_axon, vac_dend_e, vac_dend_i};
        for (int s = 0; s < 3; ++s) dst[s][t] = (uint8_t)(v[s] < 0 ? 0 : (v[s] > 255 ? 255 : v[s]));
    }
    free(bound_out);
    free(bound_in);
    free(ex_out);
    free(ex_in);
    free(del);
    free(k);
    return m;
}
