/*
 * cpu_mt.c -- multithreaded CPU baseline of the same step loop as or_run (oracle.c).
 *
 * TEST AND MEASUREMENT INFRASTRUCTURE ONLY, like the oracle: bench.py times it as a
 * second CPU baseline on all host cores, and tests/ check that it reproduces the
 * oracle's raster and state bit for bit.  The simulator library never links it.
 *
 * It includes oracle.c so that every definition (Philox, the Poisson thresholds, the
 * neuron step) is the oracle's own; only the schedule differs:
 *   - threads own contiguous neuron ranges, cut so that each range receives about
 *     the same number of synapses (in-degree), the paper's disjoint-class idea
 *     (§3.6) applied to threads;
 *   - phase 1: each thread updates its own neurons and lists its spikes; the lists
 *     are concatenated in thread order, which is ascending neuron order;
 *   - phase 2: each thread walks every spike of the step but adds only the synapses
 *     whose target it owns, from its own CSR (by sender) of those synapses, so no two
 *     threads write the same ring cell and no atomics are needed.
 * Integer addition makes the ring independent of the order of the adds, hence the
 * raster equals or_run's.  The ring is int32 here (no range report; or_run checks).
 */
#include <omp.h>
#include <stdio.h>

#include "oracle.c"

typedef struct {
    int32_t n_threads;
    int64_t N;
    int64_t *lo;          /* [T + 1] neuron range of every thread */
    int64_t **row_ptr;    /* [T][N + 1] CSR by sender of the thread's synapses */
    int32_t **post;       /* [T][...] */
    int32_t **w;
    uint8_t **d;
} mt_net;

/* Partition the oracle network's synapses by owner thread. */
void *mt_build(int32_t T, int64_t N, const int64_t *row_ptr, const int32_t *post, const int32_t *w_fx,
               const uint8_t *dly)
{
    if (T < 1) T = 1;
    mt_net *n = (mt_net *)calloc(1, sizeof(mt_net));
    if (!n) return NULL;
    n->n_threads = T;
    n->N = N;
    n->lo = (int64_t *)calloc((size_t)T + 1, sizeof(int64_t));
    n->row_ptr = (int64_t **)calloc((size_t)T, sizeof(int64_t *));
    n->post = (int32_t **)calloc((size_t)T, sizeof(int32_t *));
    n->w = (int32_t **)calloc((size_t)T, sizeof(int32_t *));
    n->d = (uint8_t **)calloc((size_t)T, sizeof(uint8_t *));
    const int64_t S = row_ptr[N];
    int64_t *indeg = (int64_t *)calloc((size_t)(N > 0 ? N : 1), sizeof(int64_t));
    int32_t *owner = (int32_t *)malloc((size_t)(N > 0 ? N : 1) * sizeof(int32_t));
    if (!n->lo || !n->row_ptr || !n->post || !n->w || !n->d || !indeg || !owner) return NULL;
    for (int64_t e = 0; e < S; ++e) indeg[post[e]] += 1;
    /* range k ends once the running in-degree reaches k/T of all synapses */
    int64_t cum = 0;
    int k = 1;
    for (int64_t i = 0; i < N; ++i) {
        owner[i] = k - 1;
        cum += indeg[i];
        while (k < T && cum * T >= (int64_t)k * S) n->lo[k++] = i + 1;
    }
    while (k <= T) n->lo[k++] = N;
    for (int t = 0; t < T; ++t)
        for (int64_t i = n->lo[t]; i < n->lo[t + 1]; ++i) owner[i] = t;
    for (int t = 0; t < T; ++t) {
        n->row_ptr[t] = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
        if (!n->row_ptr[t]) return NULL;
    }
    for (int64_t s = 0; s < N; ++s)
        for (int64_t e = row_ptr[s]; e < row_ptr[s + 1]; ++e) n->row_ptr[owner[post[e]]][s + 1] += 1;
    for (int t = 0; t < T; ++t) {
        for (int64_t s = 0; s < N; ++s) n->row_ptr[t][s + 1] += n->row_ptr[t][s];
        const int64_t St = n->row_ptr[t][N];
        n->post[t] = (int32_t *)malloc((size_t)(St > 0 ? St : 1) * sizeof(int32_t));
        n->w[t] = (int32_t *)malloc((size_t)(St > 0 ? St : 1) * sizeof(int32_t));
        n->d[t] = (uint8_t *)malloc((size_t)(St > 0 ? St : 1));
        if (!n->post[t] || !n->w[t] || !n->d[t]) return NULL;
    }
    int64_t *fill = (int64_t *)calloc((size_t)T, sizeof(int64_t));
    if (!fill) return NULL;
    for (int64_t s = 0; s < N; ++s) {
        for (int t = 0; t < T; ++t) fill[t] = n->row_ptr[t][s];
        for (int64_t e = row_ptr[s]; e < row_ptr[s + 1]; ++e) {
            const int t = owner[post[e]];
            n->post[t][fill[t]] = post[e];
            n->w[t][fill[t]] = w_fx[e];
            n->d[t][fill[t]] = dly[e];
            fill[t] += 1;
        }
    }
    free(fill);
    free(indeg);
    free(owner);
    return n;
}

void mt_free(void *p)
{
    mt_net *n = (mt_net *)p;
    if (!n) return;
    for (int t = 0; t < n->n_threads; ++t) {
        if (n->row_ptr) free(n->row_ptr[t]);
        if (n->post) free(n->post[t]);
        if (n->w) free(n->w[t]);
        if (n->d) free(n->d[t]);
    }
    free(n->row_ptr);
    free(n->post);
    free(n->w);
    free(n->d);
    free(n->lo);
    free(n);
}

/* n_steps from t0 on the thread-partitioned network; arguments and results as or_run,
 * except that W is int32.  Returns 0, or 1 if the raster capacity was exceeded. */
int mt_run(const or_model *m, uint64_t seed, const void *pn, const int64_t *pop_off, float *U, float *I,
           int32_t *R, int32_t *W, int64_t t0, int64_t n_steps, int32_t *rast_t, int32_t *rast_i,
           int64_t rast_cap, int64_t *n_rast)
{
    const mt_net *net = (const mt_net *)pn;
    const int T = net->n_threads;
    const int64_t N = net->N;
    or_lif c;
    or_lif_from_model(m, &c);
    float f[5];
    int32_t k2[2];
    or_step_constants(m, f, k2);
    const int32_t w_ext = k2[1];
    uint64_t C[OR_MAX_POPS][OR_PKMAX];
    for (int b = 0; b < m->n_pops; ++b) or_poisson_table(m, b, C[b]);
    int32_t *queue = (int32_t *)malloc((size_t)(N > 0 ? N : 1) * sizeof(int32_t));
    int64_t *cnt = (int64_t *)calloc((size_t)T + 1, sizeof(int64_t));
    if (!queue || !cnt) return -1;
    int status = 0;
    int64_t nr = *n_rast;
#pragma omp parallel num_threads(T)
    {
        const int th = omp_get_thread_num();
        const int64_t lo = net->lo[th], hi = net->lo[th + 1];
        for (int64_t t = t0; t < t0 + n_steps; ++t) {
            const int64_t slot = t % OR_DMAX;
            /* phase 1 on the own range; spikes first listed at the range start */
            int64_t nq = 0;
            int b = 0;
            while (lo >= pop_off[b + 1] && b + 1 < m->n_pops) ++b;
            for (int64_t i = lo; i < hi; ++i) {
                while (i >= pop_off[b + 1]) ++b;
                const int32_t Tn = or_poisson_count(or_poisson_uniform(seed, t, i), C[b]);
                const int32_t in = (int32_t)((uint32_t)W[slot * N + i] + (uint32_t)Tn * (uint32_t)w_ext);
                W[slot * N + i] = 0;
                if (or_neuron_step(&c, &U[i], &I[i], &R[i], in)) queue[lo + nq++] = (int32_t)i;
            }
            cnt[th + 1] = nq;
#pragma omp barrier
#pragma omp single
            {
                /* compact the per-range lists in thread (= neuron) order; record */
                int64_t q = 0;
                for (int u = 0; u < T; ++u) {
                    const int64_t n_u = cnt[u + 1];
                    memmove(queue + q, queue + net->lo[u], (size_t)n_u * sizeof(int32_t));
                    q += n_u;
                }
                cnt[0] = q;
                for (int64_t j = 0; j < q; ++j) {
                    if (nr < rast_cap) {
                        rast_t[nr] = (int32_t)t;
                        rast_i[nr] = queue[j];
                    } else {
                        status = 1;
                    }
                    ++nr;
                }
            }
            /* phase 2: this thread's synapses of every spike (implicit barrier above) */
            const int64_t *rp = net->row_ptr[th];
            const int32_t *po = net->post[th];
            const int32_t *ww = net->w[th];
            const uint8_t *dd = net->d[th];
            for (int64_t j = 0; j < cnt[0]; ++j) {
                const int64_t s = queue[j];
                for (int64_t e = rp[s]; e < rp[s + 1]; ++e) {
                    int32_t *cell = &W[((t + dd[e]) % OR_DMAX) * N + po[e]];
                    *cell = (int32_t)((uint32_t)*cell + (uint32_t)ww[e]);
                }
            }
#pragma omp barrier
        }
    }
    *n_rast = nr;
    free(queue);
    free(cnt);
    return status;
}
