/*
 * FP64 CPU oracle for Aggregate Risk Analysis (ARA).  TEST INFRASTRUCTURE ONLY:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code with the CUDA library and is deliberately plain and slow.
 *
 * What it computes (paper Section IV-B, Algorithm 3 and the prose after it):
 *   For every layer L and every trial T of the Year Event Table (Eq. 1):
 *     for every event E of T, in time order:
 *       for every ELT covered by L (Eq. 3):
 *         look E up in the ELT's direct-access table (absent event -> loss 0),
 *         apply the ELT's financial terms I = (retention R_j, limit L_j),
 *         add the result to the event's loss combined across the layer's ELTs;
 *       apply the layer's occurrence terms (OccR, OccL) to that combined loss
 *       (occurrence terms act on each occurrence on its own) and add it to the
 *       trial's aggregate loss;
 *     apply the aggregate terms (AggR, AggL) to the aggregate loss -> YLT entry.
 *
 *   Every "apply terms" step is the retention/limit clamp
 *       C(x; R, Lim) = min(max(x - R, 0), Lim)
 *   which is how this code reads the clamp printed in Section IV-B (the printed
 *   max() has lost its second argument, 0).  Limits may be +infinity.
 *
 * Everything is double precision; FP32 losses are widened exactly by the caller.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Retention/limit clamp of Section IV-B: the payout in excess of R, capped at Lim. */
static double clamp_terms(double x, double R, double Lim) {
    double excess = x - R;
    if (excess < 0.0) excess = 0.0;
    if (excess > Lim) excess = Lim;
    return excess;
}

/* Regime of the clamp at x, decided on the same excess x - R as clamp_terms:
 * 1 when 0 < x - R < Lim (slope 1 in x, -1 in R), 2 when x - R > Lim (slope 1 in Lim), else 0. */
static int clamp_regime(double x, double R, double Lim) {
    double excess = x - R;
    if (excess > 0.0 && excess < Lim) return 1;
    if (excess > Lim) return 2;
    return 0;
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * Direct-access tables (Section IV-B: "ELTs ... implemented as direct access
 * tables") for the ELTs of one layer: table[k * catalogue + e] = loss of event e
 * in the layer's k-th ELT, 0 where the ELT has no record for e.
 * Returns NULL on allocation failure or on an invalid / duplicate event ID.
 */
static double* build_tables(int64_t catalogue, int32_t n_le, const int32_t* le,
                            const int64_t* rec_off, const int32_t* rec_ids,
                            const double* rec_losses) {
    double* t = (double*)calloc((size_t)n_le * (size_t)catalogue, sizeof(double));
    unsigned char* seen = (unsigned char*)calloc((size_t)catalogue, 1);
    if (!t || !seen) { free(t); free(seen); return NULL; }
    for (int32_t k = 0; k < n_le; ++k) {
        int32_t j = le[k];
        memset(seen, 0, (size_t)catalogue);
        for (int64_t r = rec_off[j]; r < rec_off[j + 1]; ++r) {
            int32_t e = rec_ids[r];
            if (e < 0 || e >= catalogue || seen[e]) { free(t); free(seen); return NULL; }
            seen[e] = 1;
            t[(size_t)k * catalogue + e] = rec_losses[r];
        }
    }
    free(seen);
    return t;
}

/*
 * Occurrence year losses (OEP basis): for every layer and selected trial, the largest single
 * occurrence loss of the trial net of the ELT and occurrence terms, max_k o(e_k) (0 for an
 * empty trial); the aggregate terms, which act on the annual total, are not applied.
 * Same arguments and layout as orc_ylt without the aggregate outputs.
 */
int orc_ylt_oep(int64_t catalogue, const int64_t* rec_off, const int32_t* rec_ids,
                const double* rec_losses, const double* elt_ret, const double* elt_lim,
                int32_t n_layers, const int32_t* layer_off, const int32_t* layer_elts,
                const double* occ_ret, const double* occ_lim, int64_t n_trials,
                const int64_t* trial_off, const int32_t* event_ids, int64_t n_sel,
                const int64_t* sel, double* ylt_out) {
    int64_t n_out = sel ? n_sel : n_trials;
    for (int32_t l = 0; l < n_layers; ++l) {
        const int32_t* le = layer_elts + layer_off[l];
        int32_t n_le = layer_off[l + 1] - layer_off[l];
        double* tab = build_tables(catalogue, n_le, le, rec_off, rec_ids, rec_losses);
        if (!tab) return -1;
        int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(|: bad)
        for (int64_t i = 0; i < n_out; ++i) {
            int64_t t = sel ? sel[i] : i;
            if (t < 0 || t >= n_trials) { bad = 1; continue; }
            double largest = 0.0;
            for (int64_t k = trial_off[t]; k < trial_off[t + 1]; ++k) {
                int32_t e = event_ids[k];
                if (e < 0 || e >= catalogue) { bad = 1; break; }
                double l_E = 0.0;
                for (int32_t q = 0; q < n_le; ++q)
                    l_E += clamp_terms(tab[(size_t)q * catalogue + e], elt_ret[le[q]], elt_lim[le[q]]);
                double o = clamp_terms(l_E, occ_ret[l], occ_lim[l]);
                if (o > largest) largest = o;
            }
            ylt_out[(size_t)l * n_out + i] = largest;
        }
        free(tab);
        if (bad) return -1;
    }
    return 0;
}

/*
 * YLT of the selected trials for every layer.
 *   ELT records: ELT j owns records rec_off[j] .. rec_off[j+1]-1 of (rec_ids, rec_losses).
 *   Layer l covers ELTs layer_elts[layer_off[l] .. layer_off[l+1]-1], in that order.
 *   Trial t owns events trial_off[t] .. trial_off[t+1]-1 of event_ids.
 *   sel: n_sel trial indices (NULL: all n_trials trials, n_sel ignored).
 *   ylt_out[l * n_out + i]: year loss of the i-th selected trial under layer l.
 *   agg_out (may be NULL): the aggregate loss before the aggregate terms.
 * Returns 0, or -1 on bad input / allocation failure.
 */
int orc_ylt(int64_t catalogue, int32_t n_elts, const int64_t* rec_off, const int32_t* rec_ids,
            const double* rec_losses, const double* elt_ret, const double* elt_lim,
            int32_t n_layers, const int32_t* layer_off, const int32_t* layer_elts,
            const double* occ_ret, const double* occ_lim, const double* agg_ret,
            const double* agg_lim, int64_t n_trials, const int64_t* trial_off,
            const int32_t* event_ids, int64_t n_sel, const int64_t* sel,
            double* ylt_out, double* agg_out) {
    (void)n_elts;
    int64_t n_out = sel ? n_sel : n_trials;
    for (int32_t l = 0; l < n_layers; ++l) {
        const int32_t* le = layer_elts + layer_off[l];
        int32_t n_le = layer_off[l + 1] - layer_off[l];
        double* tab = build_tables(catalogue, n_le, le, rec_off, rec_ids, rec_losses);
        if (!tab) return -1;
        int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(|: bad)
        for (int64_t i = 0; i < n_out; ++i) {
            int64_t t = sel ? sel[i] : i;
            if (t < 0 || t >= n_trials) { bad = 1; continue; }
            double l_T = 0.0;                                /* the trial's aggregate loss */
            for (int64_t k = trial_off[t]; k < trial_off[t + 1]; ++k) {
                int32_t e = event_ids[k];
                if (e < 0 || e >= catalogue) { bad = 1; break; }
                double l_E = 0.0;                            /* event loss across the layer's ELTs */
                for (int32_t q = 0; q < n_le; ++q) {
                    double x = tab[(size_t)q * catalogue + e];            /* direct-access lookup */
                    l_E += clamp_terms(x, elt_ret[le[q]], elt_lim[le[q]]); /* ELT terms I */
                }
                l_T += clamp_terms(l_E, occ_ret[l], occ_lim[l]);         /* occurrence terms */
            }
            if (agg_out) agg_out[(size_t)l * n_out + i] = l_T;
            ylt_out[(size_t)l * n_out + i] = clamp_terms(l_T, agg_ret[l], agg_lim[l]);  /* aggregate */
        }
        free(tab);
        if (bad) return -1;
    }
    return 0;
}

/*
 * Gradient of J_l = sum_t w[l * n_trials + t] * y_{l,t} for every layer l, by the chain rule
 * applied occurrence by occurrence through the same loops as orc_ylt.  The clamp
 * C(x; R, Lim) has dC/dx = [0 < x-R < Lim], dC/dR = -[0 < x-R < Lim], dC/dLim = [x-R > Lim]
 * (strict inequalities: the derivative at a kink is taken as 0).
 * Outputs, per layer l (caller zero-fills nothing; this routine overwrites):
 *   g_elt[l][k][0..1]  = dJ/dR_j, dJ/dLim_j for the layer's k-th ELT j   (layout [layer_off[n_layers]][2])
 *   g_layer[l][0..3]   = dJ/dOccR, dJ/dOccL, dJ/dAggR, dJ/dAggL
 *   g_loss[rec_pos]    = dJ/dx for every record of every ELT of the layer, laid out per layer
 *                        as the concatenation of its ELTs' records (layout given by g_loss_off[l]).
 */
int orc_adjoint(int64_t catalogue, const int64_t* rec_off, const int32_t* rec_ids,
                const double* rec_losses, const double* elt_ret, const double* elt_lim,
                int32_t n_layers, const int32_t* layer_off, const int32_t* layer_elts,
                const double* occ_ret, const double* occ_lim, const double* agg_ret,
                const double* agg_lim, int64_t n_trials, const int64_t* trial_off,
                const int32_t* event_ids, const double* w, double* g_elt, double* g_layer,
                const int64_t* g_loss_off, double* g_loss) {
    for (int32_t l = 0; l < n_layers; ++l) {
        const int32_t* le = layer_elts + layer_off[l];
        int32_t n_le = layer_off[l + 1] - layer_off[l];
        double* tab = build_tables(catalogue, n_le, le, rec_off, rec_ids, rec_losses);
        double* gx = (double*)calloc((size_t)n_le * (size_t)catalogue, sizeof(double));
        double* gR = (double*)calloc((size_t)n_le, sizeof(double));
        double* gL = (double*)calloc((size_t)n_le, sizeof(double));
        if (!tab || !gx || !gR || !gL) { free(tab); free(gx); free(gR); free(gL); return -1; }
        double oR = occ_ret[l], oL = occ_lim[l], aR = agg_ret[l], aL = agg_lim[l];
        double g_occR = 0.0, g_occL = 0.0, g_aggR = 0.0, g_aggL = 0.0;
        for (int64_t t = 0; t < n_trials; ++t) {
            double wt = w[(size_t)l * n_trials + t];
            if (wt == 0.0) continue;
            /* forward for this trial */
            double l_T = 0.0;
            for (int64_t k = trial_off[t]; k < trial_off[t + 1]; ++k) {
                int32_t e = event_ids[k];
                double l_E = 0.0;
                for (int32_t q = 0; q < n_le; ++q)
                    l_E += clamp_terms(tab[(size_t)q * catalogue + e], elt_ret[le[q]], elt_lim[le[q]]);
                l_T += clamp_terms(l_E, oR, oL);
            }
            /* dy/dl_T and the aggregate terms */
            int agg = clamp_regime(l_T, aR, aL);
            if (agg == 1) g_aggR -= wt;
            if (agg == 2) g_aggL += wt;
            if (agg != 1) continue;
            /* back through every occurrence */
            for (int64_t k = trial_off[t]; k < trial_off[t + 1]; ++k) {
                int32_t e = event_ids[k];
                double l_E = 0.0;
                for (int32_t q = 0; q < n_le; ++q)
                    l_E += clamp_terms(tab[(size_t)q * catalogue + e], elt_ret[le[q]], elt_lim[le[q]]);
                int occ = clamp_regime(l_E, oR, oL);
                if (occ == 1) g_occR -= wt;
                if (occ == 2) g_occL += wt;
                if (occ != 1) continue;
                for (int32_t q = 0; q < n_le; ++q) {
                    double x = tab[(size_t)q * catalogue + e];
                    int reg = clamp_regime(x, elt_ret[le[q]], elt_lim[le[q]]);
                    if (reg == 1) {
                        gx[(size_t)q * catalogue + e] += wt;
                        gR[q] -= wt;
                    }
                    if (reg == 2) gL[q] += wt;
                }
            }
        }
        for (int32_t q = 0; q < n_le; ++q) {
            g_elt[((size_t)layer_off[l] + q) * 2 + 0] = gR[q];
            g_elt[((size_t)layer_off[l] + q) * 2 + 1] = gL[q];
        }
        g_layer[(size_t)l * 4 + 0] = g_occR;
        g_layer[(size_t)l * 4 + 1] = g_occL;
        g_layer[(size_t)l * 4 + 2] = g_aggR;
        g_layer[(size_t)l * 4 + 3] = g_aggL;
        int64_t pos = g_loss_off[l];
        for (int32_t q = 0; q < n_le; ++q) {
            int32_t j = le[q];
            for (int64_t r = rec_off[j]; r < rec_off[j + 1]; ++r)
                g_loss[pos++] = gx[(size_t)q * catalogue + rec_ids[r]];
        }
        free(tab); free(gx); free(gR); free(gL);
    }
    return 0;
}
