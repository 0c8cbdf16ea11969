/* msp_neuron.h -- oracle of the Model of Structural Plasticity's neuron side
 * (Section 3.1, Table 1): electrical activity (Poisson spiking), calcium,
 * synaptic-element growth and synapse deletion, which together produce the
 * vacant elements the synapse search consumes.
 *
 * TEST INFRASTRUCTURE ONLY (see msp_oracle.h).
 *
 * Precision: the paper fixes none.  The neuron state decides integers (a
 * spike, the floor of an element count), so the oracle computes it in single
 * precision with every operation in the stated order (no contraction), the
 * precision of the kernels; exp is computed by orc_expf below, written from
 * its definition, so both sides round identically.
 */
#ifndef MSP_NEURON_ORACLE_H
#define MSP_NEURON_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Table 1 parameters (and the refractory period and the input per spiking
 * presynaptic neuron of Section 3.1). */
typedef struct {
    float x0;              /* resting potential, 0.05                       */
    float tau_x;           /* membrane potential decay constant, 5          */
    float background;      /* background activity per step, 0.003           */
    float input_per_spike; /* per spiking presynaptic partner, 5e-4         */
    int   refractory;      /* steps without a spike after one, 4            */
    float beta_ca;         /* calcium increase per spike, 5e-4 (Table 1)    */
    float decay_ca;        /* calcium decay per step, 1e-5                  */
    float eps;             /* growth curve right intersection, 0.7          */
    float eta_axon;        /* left intersection, axons, 0.4                 */
    float eta_dend;        /* left intersection, dendrites, 0.1             */
    float mu;              /* growth scaling (maximum rate), 1e-4           */
} orc_neuron_params;

/* exp(x) for x <= 0 in single precision: Cody and Waite's range reduction
 * x = n ln2 + r (ln2 split in two parts) and the Taylor polynomial of e^r to
 * degree 7, scaled by 2^n; 0 below -87. */
float orc_expf(float x);

/* Growth of synaptic elements per step at calcium ca (Gaussian growth curve
 * of the cited model: zero at ca = eta and ca = eps, maximum mu halfway). */
float orc_growth(float ca, float eta, float eps, float mu);

/* n_steps simulation steps first_step, first_step+1, ...  Per step: the
 * input of neuron t is the number of edges s -> t whose s spiked in the
 * previous step (spiked[] on entry); then activity, spike, calcium and
 * elements as in Section 3.1.  spiked[] holds the last step's spikes on
 * return. */
void orc_neuron_steps(int64_t n, uint64_t seed, uint64_t first_step, int n_steps,
                      const orc_neuron_params *mp, int64_t n_edges, const int32_t *edge_pre,
                      const int32_t *edge_post, float *x, uint8_t *refractory, float *calcium,
                      float *z_axon, float *z_dend_e, float *z_dend_i, uint8_t *spiked);

/* Synapse deletion and vacancies (Section 3.1, update of synapses).  A neuron
 * with more bound synapses than floor(elements) on a side deletes the excess,
 * chosen uniformly at random (the excess edges with the smallest Philox
 * priorities, ties by edge position); an edge chosen by either side is
 * removed.  The edge list is compacted in place, order kept; returns the new
 * edge count.  Then vacant = floor(elements) - bound synapses, clamped to
 * [0, 255]. */
int64_t orc_update_synapses(int64_t n, uint64_t seed, uint64_t step, const float *z_axon,
                            const float *z_dend_e, const float *z_dend_i, int64_t n_edges,
                            int32_t *edge_pre, int32_t *edge_post, uint8_t *edge_type,
                            uint8_t *vac_axon, uint8_t *vac_dend_e, uint8_t *vac_dend_i);

#ifdef __cplusplus
}
#endif

#endif
