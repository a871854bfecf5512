/*
 * oracle.c -- plain, slow, single-threaded CPU oracle of the Potjans-Diesmann
 * microcircuit step loop of Lindqvist & Podobas, "Fast Algorithms for Spiking
 * Neural Network Simulation with FPGAs" (arXiv 2405.02019).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the simulator library links, includes or
 * calls this file; only the tests, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg load it (through oracle/__init__.py).  It shares no code, header,
 * table or constant with the CUDA path: every quantity below is derived here again
 * from the paper's equations and the readings stated with each function.
 *
 * Arithmetic rules: FP64 for host constants and network sampling; the neuron state
 * is FP32 with every product and sum rounded separately (build with
 * -ffp-contract=off; no FMA); synaptic input is accumulated exactly in int64 and
 * handed to the neuron as an int32 count of 2^-12 pA (the reading of §4.1's
 * remark that FP32 accumulation order changes results: an integer sum has one
 * correct value).
 *
 * Parity status: every function here is pinned by a test in tests/ against the
 * paper's printed values, closed forms or an external library (numpy's Philox,
 * scipy's Poisson CDF), except the full network dynamics, for which the paper
 * prints no reproducible numbers (parity of whole rasters is GPU-vs-oracle only).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_POPS 8
#define OR_MAX_OVR 4
#define OR_DMAX 64      /* rows of the wrap-around ring W (§3.2): a power of two > max delay */
#define OR_FX_SHIFT 12  /* one unit of synaptic input = 2^-12 pA */
#define OR_PKMAX 24     /* length of a Poisson threshold table */

/* One circuit's parameters; field order must match oracle/__init__.py. */
typedef struct {
    int32_t n_pops;
    int32_t n_ovr;
    double dt_ms, C_m_pF, tau_m_ms, tau_ref_ms, tau_syn_ms;
    double u_rest_mV, u_reset_mV, u_thr_mV, nu_th_hz, w_ext_mV;
    int64_t n_full[OR_MAX_POPS];
    double k_ext[OR_MAX_POPS];
    double u0_mean[OR_MAX_POPS], u0_sd[OR_MAX_POPS];
    double w_mean[OR_MAX_POPS], w_sd[OR_MAX_POPS];
    double d_mean[OR_MAX_POPS], d_sd[OR_MAX_POPS];
    double conn_p[OR_MAX_POPS][OR_MAX_POPS]; /* [target][source] */
    int32_t ovr_src[OR_MAX_OVR], ovr_tgt[OR_MAX_OVR];
    double ovr_mean[OR_MAX_OVR], ovr_sd[OR_MAX_OVR];
} or_model;

/* Stream tags (second Philox key word) of the three random streams. */
#define OR_TAG_CONN 0xC0u
#define OR_TAG_INIT 0x1Au
#define OR_TAG_POIS 0x7Au

/* ------------------------------------------------------------------------ */
/* Philox4x64-10, from its publication: Salmon, Moraes, Dror, Shaw, "Parallel   */
/* random numbers: as easy as 1, 2, 3", SC'11.  One round multiplies counter   */
/* words 0 and 2 by two odd constants, and permutes high/low halves xored with */
/* the other counter words and the key; the key is bumped by two Weyl          */
/* constants between rounds.                                                   */
/* ------------------------------------------------------------------------ */
static void or_mul128(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void or_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t hi0, lo0, hi1, lo1;
        or_mul128(M0, c0, &hi0, &lo0);
        or_mul128(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform double in (0, 1) from the top 53 bits of a 64-bit word. */
static double or_unit(uint64_t x)
{
    return ((double)(x >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/* Box-Muller (Box & Muller 1958): two independent standard normals from two
 * uniforms u, v: r = sqrt(-2 ln u), z_cos = r cos(2 pi v), z_sin = r sin(2 pi v). */
static void or_box_muller(uint64_t a, uint64_t b, double *z_cos, double *z_sin)
{
    double r = sqrt(-2.0 * log(or_unit(a)));
    double th = 6.283185307179586 * or_unit(b);
    *z_cos = r * cos(th);
    *z_sin = r * sin(th);
}

/* High 64 bits of x * n: a uniform integer in [0, n) from a uniform 64-bit x. */
static int64_t or_below(uint64_t x, int64_t n)
{
    uint64_t hi, lo;
    or_mul128(x, (uint64_t)n, &hi, &lo);
    return (int64_t)hi;
}

/* ------------------------------------------------------------------------ */
/* Host constants (§2.2, the equations for w_f, p11, p22, beta, gamma, p21).   */
/* out: w_f [pA/mV], p11, p22, beta [ms], gamma [ms/pF], p21 [mV/pA].          */
/* ------------------------------------------------------------------------ */
void or_constants(const or_model *m, double out[6])
{
    const double ts = m->tau_syn_ms, tm = m->tau_m_ms, C = m->C_m_pF, dt = m->dt_ms;
    /* PSP-to-PSC factor: d = tau_syn - tau_m, p = tau_syn tau_m, q = tau_m / tau_syn,
       w_f = C_m d / (p (q^(tau_m/d) - q^(tau_syn/d))). */
    const double d = ts - tm;
    const double p = ts * tm;
    const double q = tm / ts;
    const double w_f = C * d / (p * (pow(q, tm / d) - pow(q, ts / d)));
    /* Decay of the synaptic current and of the membrane over one step. */
    const double p11 = exp(-dt / ts);
    const double p22 = exp(-dt / tm);
    /* Injection of the synaptic current into the membrane over one step. */
    const double beta = ts * tm / (tm - ts);
    const double gamma = beta / C;
    const double p21 = p11 * gamma * (exp(dt / beta) - 1.0);
    out[0] = w_f; out[1] = p11; out[2] = p22; out[3] = beta; out[4] = gamma; out[5] = p21;
}

/* The FP32 / integer constants the step loop uses.
 * fout: p11, p21, p22, theta (u_thr - u_rest), u_reset - u_rest  (all mV / pA, FP32)
 * iout: t_ref in steps (tau_ref / dt rounded), thalamic weight in 2^-12 pA units
 *       (w_f * omega_ext scaled by 2^12 and rounded). */
void or_step_constants(const or_model *m, float fout[5], int32_t iout[2])
{
    double c[6];
    or_constants(m, c);
    fout[0] = (float)c[1];
    fout[1] = (float)c[5];
    fout[2] = (float)c[2];
    fout[3] = (float)(m->u_thr_mV - m->u_rest_mV);
    fout[4] = (float)(m->u_reset_mV - m->u_rest_mV);
    iout[0] = (int32_t)llround(m->tau_ref_ms / m->dt_ms);
    iout[1] = (int32_t)llround(c[0] * m->w_ext_mV * 4096.0);
}

/* ------------------------------------------------------------------------ */
/* Network size (Table params2 N_i, §2.2) at an integer permille scale,        */
/* rounded half up; populations are laid out contiguously in table order.      */
/* ------------------------------------------------------------------------ */
void or_pop_sizes(const or_model *m, int32_t scale_n, int64_t out[OR_MAX_POPS])
{
    for (int b = 0; b < m->n_pops; ++b)
        out[b] = (m->n_full[b] * (int64_t)scale_n + 500) / 1000;
}

/* Number of synapses from source population a to target population b: the
 * paper's expected count N_pre * N_post * p (§2.2, the L23/inh -> L5/exc example),
 * with the source count scaled by the in-degree scale and the target count by the
 * neuron scale, rounded to the nearest integer. */
int64_t or_pair_count(const or_model *m, int32_t scale_n, int32_t scale_k, int32_t b, int32_t a)
{
    int64_t nb[OR_MAX_POPS];
    or_pop_sizes(m, scale_n, nb);
    const double src = (double)(m->n_full[a] * (int64_t)scale_k) / 1000.0;
    return (int64_t)llround(m->conn_p[b][a] * src * (double)nb[b]);
}

int64_t or_total_synapses(const or_model *m, int32_t scale_n, int32_t scale_k)
{
    int64_t s = 0;
    for (int a = 0; a < m->n_pops; ++a)
        for (int b = 0; b < m->n_pops; ++b)
            s += or_pair_count(m, scale_n, scale_k, b, a);
    return s;
}

/* Mean/SD of the amplitude (mV) of a synapse from a to b: the source population's
 * row of Table params2, replaced by an override for listed (a, b) pairs. */
static void or_weight_law(const or_model *m, int a, int b, double *mu, double *sd)
{
    *mu = m->w_mean[a];
    *sd = m->w_sd[a];
    for (int o = 0; o < m->n_ovr; ++o)
        if (m->ovr_src[o] == a && m->ovr_tgt[o] == b) {
            *mu = m->ovr_mean[o];
            *sd = m->ovr_sd[o];
        }
}

/* ------------------------------------------------------------------------ */
/* One synapse, k-th of pair (a -> b), drawn with replacement (§2.2: multapses  */
/* and autapses allowed).  One Philox call, key (seed, CONN), counter (k, a, b,  */
/* 0): word 0 picks the source neuron, word 1 the target, words 2-3 give a      */
/* Box-Muller pair whose cosine branch sets the amplitude and sine branch the   */
/* delay.  Amplitude in mV is mapped to current with w_f, clipped at zero on    */
/* the wrong side of its sign, and stored as an integer count of 2^-12 pA       */
/* (w_pA, when not NULL, receives the current before that rounding).           */
/* Delay in ms is rounded to whole steps and clipped to [1, DMAX-1].            */
/* ------------------------------------------------------------------------ */
static void or_draw_synapse(const or_model *m, uint64_t seed, double w_f, const int64_t *off,
                            const int64_t *nb, int a, int b, int64_t k,
                            int32_t *pre, int32_t *post, int32_t *w_fx, double *w_pA, uint8_t *dly)
{
    uint64_t ctr[4] = {(uint64_t)k, (uint64_t)a, (uint64_t)b, 0};
    uint64_t key[2] = {seed, OR_TAG_CONN};
    uint64_t u[4];
    or_philox4x64_10(ctr, key, u);
    *pre = (int32_t)(off[a] + or_below(u[0], nb[a]));
    *post = (int32_t)(off[b] + or_below(u[1], nb[b]));
    double zw, zd;
    or_box_muller(u[2], u[3], &zw, &zd);
    double mu, sd;
    or_weight_law(m, a, b, &mu, &sd);
    double w_mV = mu + sd * zw;
    if (mu >= 0.0 && w_mV < 0.0) w_mV = 0.0;
    if (mu < 0.0 && w_mV > 0.0) w_mV = 0.0;
    const double amp_pA = w_mV * w_f;
    *w_fx = (int32_t)llround(amp_pA * 4096.0);
    if (w_pA) *w_pA = amp_pA;
    double d_ms = m->d_mean[a] + m->d_sd[a] * zd;
    long long ds = llround(d_ms / m->dt_ms);
    if (ds < 1) ds = 1;
    if (ds > OR_DMAX - 1) ds = OR_DMAX - 1;
    *dly = (uint8_t)ds;
}

/* Build the network: every synapse of every pair, then grouped by source neuron
 * (a stable counting sort: within a row, synapses keep generation order) so that
 * "syns_from(i)" of Listing push is the contiguous slice row_ptr[i]..row_ptr[i+1]
 * (§3.5).  Outputs are caller-allocated: row_ptr[N+1], post/w_fx/dly[S], and, when
 * w_pA is not NULL, w_pA[S]: the same synapses' currents in pA before rounding to
 * 2^-12 pA (the weights of the FP64 reference loop).
 * Returns 0, or -1 on allocation failure. */
int or_build(const or_model *m, int32_t scale_n, int32_t scale_k, uint64_t seed,
             int64_t *row_ptr, int32_t *post, int32_t *w_fx, uint8_t *dly, double *w_pA)
{
    int64_t nb[OR_MAX_POPS], off[OR_MAX_POPS + 1];
    or_pop_sizes(m, scale_n, nb);
    off[0] = 0;
    for (int b = 0; b < m->n_pops; ++b) off[b + 1] = off[b] + nb[b];
    const int64_t N = off[m->n_pops];
    const int64_t S = or_total_synapses(m, scale_n, scale_k);
    double c[6];
    or_constants(m, c);

    int32_t *g_pre = (int32_t *)malloc((size_t)(S > 0 ? S : 1) * sizeof(int32_t));
    int32_t *g_post = (int32_t *)malloc((size_t)(S > 0 ? S : 1) * sizeof(int32_t));
    int32_t *g_w = (int32_t *)malloc((size_t)(S > 0 ? S : 1) * sizeof(int32_t));
    uint8_t *g_d = (uint8_t *)malloc((size_t)(S > 0 ? S : 1));
    double *g_a = w_pA ? (double *)malloc((size_t)(S > 0 ? S : 1) * sizeof(double)) : NULL;
    if (!g_pre || !g_post || !g_w || !g_d || (w_pA && !g_a)) {
        free(g_pre); free(g_post); free(g_w); free(g_d); free(g_a);
        return -1;
    }
    int64_t s = 0;
    for (int a = 0; a < m->n_pops; ++a)
        for (int b = 0; b < m->n_pops; ++b) {
            const int64_t K = or_pair_count(m, scale_n, scale_k, b, a);
            for (int64_t k = 0; k < K; ++k, ++s)
                or_draw_synapse(m, seed, c[0], off, nb, a, b, k, &g_pre[s], &g_post[s], &g_w[s],
                                g_a ? &g_a[s] : NULL, &g_d[s]);
        }
    /* counting sort by source neuron */
    for (int64_t i = 0; i <= N; ++i) row_ptr[i] = 0;
    for (int64_t k = 0; k < S; ++k) row_ptr[g_pre[k] + 1] += 1;
    for (int64_t i = 0; i < N; ++i) row_ptr[i + 1] += row_ptr[i];
    int64_t *fill = (int64_t *)malloc((size_t)(N > 0 ? N : 1) * sizeof(int64_t));
    if (!fill) {
        free(g_pre); free(g_post); free(g_w); free(g_d); free(g_a);
        return -1;
    }
    for (int64_t i = 0; i < N; ++i) fill[i] = row_ptr[i];
    for (int64_t k = 0; k < S; ++k) {
        int64_t dst = fill[g_pre[k]]++;
        post[dst] = g_post[k];
        w_fx[dst] = g_w[k];
        dly[dst] = g_d[k];
        if (g_a) w_pA[dst] = g_a[k];
    }
    free(fill);
    free(g_pre); free(g_post); free(g_w); free(g_d); free(g_a);
    return 0;
}

/* Initial membrane potential (Table params2, column u_init), relative to rest:
 * neuron i (circuit-local index) draws Philox key (seed, INIT), counter
 * (i, 0, 0, 0); Box-Muller's cosine branch of words 0-1 gives z, and
 * U = (float)(mu + sd z - u_rest). */
void or_initial_u(const or_model *m, int32_t scale_n, uint64_t seed, float *U)
{
    int64_t nb[OR_MAX_POPS];
    or_pop_sizes(m, scale_n, nb);
    int64_t i = 0;
    for (int b = 0; b < m->n_pops; ++b)
        for (int64_t j = 0; j < nb[b]; ++j, ++i) {
            uint64_t ctr[4] = {(uint64_t)i, 0, 0, 0};
            uint64_t key[2] = {seed, OR_TAG_INIT};
            uint64_t u[4];
            or_philox4x64_10(ctr, key, u);
            double zc, zs;
            or_box_muller(u[0], u[1], &zc, &zs);
            U[i] = (float)(m->u0_mean[b] + m->u0_sd[b] * zc - m->u_rest_mV);
        }
}

/* ------------------------------------------------------------------------ */
/* Thalamic drive (§2.2, Eq. psc and the sentence after Eq. ref): T_t of a      */
/* neuron of population b is Poisson with mean nu_th K_b dt.  The draw is by    */
/* inversion of the CDF: with the Poisson pmf built by its recurrence           */
/* pmf_0 = e^-lambda, pmf_k = pmf_{k-1} lambda / k and F_k = F_{k-1} + pmf_k,   */
/* thresholds C_k = floor(F_k 2^63) (2^63 once F_k >= 1), and T = #{k : v >=   */
/* C_k} for a uniform 63-bit v.                                                 */
/* ------------------------------------------------------------------------ */
void or_poisson_table(const or_model *m, int32_t pop, uint64_t out[OR_PKMAX])
{
    const double lam = m->k_ext[pop] * m->nu_th_hz * m->dt_ms * 1e-3;
    double pmf = exp(-lam);
    double F = pmf;
    for (int k = 0; k < OR_PKMAX; ++k) {
        if (k > 0) {
            pmf = pmf * lam / (double)k;
            F = F + pmf;
        }
        if (k == OR_PKMAX - 1 || F >= 1.0)
            out[k] = 9223372036854775808ULL;
        else
            out[k] = (uint64_t)(F * 9223372036854775808.0);
    }
}

/* The uniform of neuron i (circuit-local) at step t: word (i mod 4) of Philox
 * key (seed, POIS), counter (t, i / 4, 0, 0), shifted to 63 bits. */
static uint64_t or_poisson_uniform(uint64_t seed, int64_t t, int64_t i)
{
    uint64_t ctr[4] = {(uint64_t)t, (uint64_t)(i >> 2), 0, 0};
    uint64_t key[2] = {seed, OR_TAG_POIS};
    uint64_t u[4];
    or_philox4x64_10(ctr, key, u);
    return u[i & 3] >> 1;
}

static int32_t or_poisson_count(uint64_t v, const uint64_t C[OR_PKMAX])
{
    int32_t T = 0;
    for (int k = 0; k < OR_PKMAX; ++k)
        if (v >= C[k]) T += 1;
    return T;
}

/* T for a given 63-bit uniform v and population `pop`: the inversion count of the
 * table above (pins its boundaries without a random draw). */
int32_t or_poisson_count_at(const or_model *m, int32_t pop, uint64_t v)
{
    uint64_t C[OR_PKMAX];
    or_poisson_table(m, pop, C);
    return or_poisson_count(v, C);
}

/* n draws for neurons i0..i0+n-1 (all taken as population `pop`) at step t. */
void or_poisson_draws(const or_model *m, uint64_t seed, int32_t pop, int64_t t, int64_t i0,
                      int64_t n, int32_t *out)
{
    uint64_t C[OR_PKMAX];
    or_poisson_table(m, pop, C);
    for (int64_t j = 0; j < n; ++j) out[j] = or_poisson_count(or_poisson_uniform(seed, t, i0 + j), C);
}

/* ------------------------------------------------------------------------ */
/* One neuron, one step: Listing push (§3.1) with Eqs. mem, psc, ref (§2.2).    */
/* If not refractory, u <- p22 u + p21 I; reaching theta is a spike: u is reset */
/* and r <- t_ref.  If refractory, u stays at reset and r counts down.  Then    */
/* I <- p11 I + (thalamic + recurrent input arriving this step).  Every FP32    */
/* product and sum is rounded on its own.  Returns 1 on a spike.                */
/* ------------------------------------------------------------------------ */
typedef struct {
    float p11, p21, p22, theta, u_reset;
    int32_t t_ref;
} or_lif;

static int or_neuron_step(const or_lif *c, float *U, float *I, int32_t *R, int32_t in_fx)
{
    int spike = 0;
    if (*R == 0) {
        float a = c->p22 * *U;
        float b = c->p21 * *I;
        float x = a + b;
        if (x >= c->theta) {
            spike = 1;
            x = c->u_reset;
            *R = c->t_ref;
        }
        *U = x;
    } else {
        *U = c->u_reset;
        *R -= 1;
    }
    float decayed = c->p11 * *I;
    float arriving = (float)in_fx * (1.0f / 4096.0f);
    *I = decayed + arriving;
    return spike;
}

static void or_lif_from_model(const or_model *m, or_lif *c)
{
    float f[5];
    int32_t k[2];
    or_step_constants(m, f, k);
    c->p11 = f[0]; c->p21 = f[1]; c->p22 = f[2]; c->theta = f[3]; c->u_reset = f[4];
    c->t_ref = k[0];
}

/* A single neuron driven by a given input sequence in_fx[0..n) (2^-12 pA units).
 * Writes the state after every step and the spike flags.  Uses exactly the update
 * of or_run. */
void or_lif_trace(const or_model *m, float U0, float I0, int32_t R0, int64_t n, const int32_t *in_fx,
                  float *U_out, float *I_out, int32_t *R_out, int32_t *spk_out)
{
    or_lif c;
    or_lif_from_model(m, &c);
    float U = U0, I = I0;
    int32_t R = R0;
    for (int64_t t = 0; t < n; ++t) {
        spk_out[t] = or_neuron_step(&c, &U, &I, &R, in_fx[t]);
        U_out[t] = U;
        I_out[t] = I;
        R_out[t] = R;
    }
}

/* ------------------------------------------------------------------------ */
/* n_steps of the network, starting at step t0 (Listing push, deferred as in   */
/* Listing push2, ring indexed modulo DMAX as in §3.2).                          */
/*                                                                              */
/* Phase 1, every neuron i in index order: the neuron step of or_neuron_step    */
/* with input W[t mod DMAX][i] + T(t, i) * w_ext; the ring cell is cleared       */
/* after the read.  Spikes are recorded as (t, i) and queued.                    */
/* Phase 2, every queued neuron s in ascending order: each synapse (j, d, w) of  */
/* row s adds w to W[(t + d) mod DMAX][j].                                       */
/*                                                                              */
/* The ring holds exact int64 sums; an input whose value leaves the int32 range */
/* is reported (return 2), since a fixed-point path could not represent it.     */
/* pop_off[n_pops+1] gives each neuron's population for its Poisson table.      */
/* State U, I, R (R in steps) and W[DMAX*N] are read and updated in place.      */
/* Returns 0, 1 if the raster capacity was exceeded, 2 on an int32 range error, */
/* -1 on allocation failure.                                                    */
/* ------------------------------------------------------------------------ */
int or_run(const or_model *m, uint64_t seed, int64_t N, const int64_t *pop_off,
           const int64_t *row_ptr, const int32_t *post, const int32_t *w_fx, const uint8_t *dly,
           float *U, float *I, int32_t *R, int64_t *W, int64_t t0, int64_t n_steps,
           int32_t *rast_t, int32_t *rast_i, int64_t rast_cap, int64_t *n_rast)
{
    or_lif c;
    or_lif_from_model(m, &c);
    float f[5];
    int32_t k2[2];
    or_step_constants(m, f, k2);
    const int64_t w_ext = k2[1];
    uint64_t C[OR_MAX_POPS][OR_PKMAX];
    for (int b = 0; b < m->n_pops; ++b) or_poisson_table(m, b, C[b]);

    int32_t *queue = (int32_t *)malloc((size_t)(N > 0 ? N : 1) * sizeof(int32_t));
    if (!queue) return -1;
    int status = 0;
    int64_t nr = *n_rast;
    for (int64_t t = t0; t < t0 + n_steps; ++t) {
        const int64_t slot = t % OR_DMAX;
        int64_t nq = 0;
        int b = 0;
        for (int64_t i = 0; i < N; ++i) {
            while (i >= pop_off[b + 1]) ++b;
            const int32_t T = or_poisson_count(or_poisson_uniform(seed, t, i), C[b]);
            const int64_t in = W[slot * N + i] + (int64_t)T * w_ext;
            W[slot * N + i] = 0;
            if (in > INT32_MAX || in < INT32_MIN) status = 2;
            if (or_neuron_step(&c, &U[i], &I[i], &R[i], (int32_t)in)) {
                queue[nq++] = (int32_t)i;
                if (nr < rast_cap) {
                    rast_t[nr] = (int32_t)t;
                    rast_i[nr] = (int32_t)i;
                } else if (status == 0) {
                    status = 1;
                }
                ++nr;
            }
        }
        for (int64_t q = 0; q < nq; ++q) {
            const int64_t s = queue[q];
            for (int64_t e = row_ptr[s]; e < row_ptr[s + 1]; ++e) {
                const int64_t slot2 = (t + dly[e]) % OR_DMAX;
                W[slot2 * N + post[e]] += w_fx[e];
            }
        }
    }
    *n_rast = nr;
    free(queue);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Compressed synapse records (reduced-precision weights, §5.3): the weights a  */
/* compressed store reproduces, computed here from their definitions.           */
/* ------------------------------------------------------------------------ */

static int or_pop_of(int32_t n_pops, const int64_t *pop_off, int64_t i)
{
    int b = 0;
    while (b + 1 < n_pops && i >= pop_off[b + 1]) ++b;
    return b;
}

/* int8 codes with one affine scale per (source population, target population)
 * pair, fitted to the pair's weights ("deviation from the mean" storage): with lo,
 * hi the pair's smallest and largest weight, base = lo + (hi - lo) div 2 and step =
 * max(1, ceil((hi - lo) / 254)); a weight w becomes q = clamp(round((w - base) /
 * step), -127, 127) and reads back as base + q step.  Rows are given as the CSR of
 * the network (row i = source neuron i).  Writes the read-back weights to w_out and
 * the [8][8] tables to base_out / step_out. */
void or_quantize_i8(int32_t n_pops, const int64_t *pop_off, int64_t N, const int64_t *row_ptr, const int32_t *post,
                    const int32_t *w_fx, int32_t *w_out, int32_t *base_out, int32_t *step_out)
{
    int64_t lo[OR_MAX_POPS][OR_MAX_POPS], hi[OR_MAX_POPS][OR_MAX_POPS];
    int seen[OR_MAX_POPS][OR_MAX_POPS];
    memset(seen, 0, sizeof(seen));
    for (int64_t i = 0; i < N; ++i) {
        const int a = or_pop_of(n_pops, pop_off, i);
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int b = or_pop_of(n_pops, pop_off, post[e]);
            if (!seen[a][b] || w_fx[e] < lo[a][b]) lo[a][b] = w_fx[e];
            if (!seen[a][b] || w_fx[e] > hi[a][b]) hi[a][b] = w_fx[e];
            seen[a][b] = 1;
        }
    }
    for (int a = 0; a < OR_MAX_POPS; ++a)
        for (int b = 0; b < OR_MAX_POPS; ++b) {
            int64_t base = 0, step = 1;
            if (a < n_pops && b < n_pops && seen[a][b]) {
                base = lo[a][b] + (hi[a][b] - lo[a][b]) / 2;
                step = (hi[a][b] - lo[a][b] + 253) / 254;
                if (step < 1) step = 1;
            }
            base_out[a * OR_MAX_POPS + b] = (int32_t)base;
            step_out[a * OR_MAX_POPS + b] = (int32_t)step;
        }
    for (int64_t i = 0; i < N; ++i) {
        const int a = or_pop_of(n_pops, pop_off, i);
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int b = or_pop_of(n_pops, pop_off, post[e]);
            const int64_t base = base_out[a * OR_MAX_POPS + b], step = step_out[a * OR_MAX_POPS + b];
            long long q = llround((double)(w_fx[e] - base) / (double)step);
            if (q > 127) q = 127;
            if (q < -127) q = -127;
            w_out[e] = (int32_t)(base + q * step);
        }
    }
}

/* bfloat16 currents: the weight in pA (w_fx 2^-12) as a float, rounded to 8
 * significand bits with ties to even, read back in 2^-12 pA units (exact). */
void or_quantize_bf16(int64_t S, const int32_t *w_fx, int32_t *w_out)
{
    for (int64_t e = 0; e < S; ++e) {
        float f = (float)w_fx[e] * (1.0f / 4096.0f);
        uint32_t u;
        memcpy(&u, &f, 4);
        const uint32_t lsb = (u >> 16) & 1u;
        u = (u + 0x7FFFu + lsb) & 0xFFFF0000u;
        float g;
        memcpy(&g, &u, 4);
        w_out[e] = (int32_t)(g * 4096.0f);
    }
}

/* The step loop of or_run in FP64 throughout (the reference for the accuracy of the
 * FP32 and compressed forms): FP64 neuron state and propagators, synaptic weights
 * w_pA in pA as drawn (before any rounding to 2^-12 pA), the thalamic amplitude
 * w_f w_ext in pA, and a double ring W[DMAX*N] that sums the currents in pA.
 * The spike order, delays and Poisson draws are those of or_run. */
int or_run_f64(const or_model *m, uint64_t seed, int64_t N, const int64_t *pop_off, const int64_t *row_ptr,
               const int32_t *post, const double *w_pA, const uint8_t *dly, double *U, double *I, int32_t *R,
               double *W, int64_t t0, int64_t n_steps, int32_t *rast_t, int32_t *rast_i, int64_t rast_cap,
               int64_t *n_rast)
{
    double c[6];
    or_constants(m, c);
    const double p11 = c[1], p22 = c[2], p21 = c[5];
    const double theta = m->u_thr_mV - m->u_rest_mV, u_reset = m->u_reset_mV - m->u_rest_mV;
    float f[5];
    int32_t k2[2];
    or_step_constants(m, f, k2);
    const int32_t t_ref = k2[0];
    const double w_ext = c[0] * m->w_ext_mV;
    uint64_t C[OR_MAX_POPS][OR_PKMAX];
    for (int b = 0; b < m->n_pops; ++b) or_poisson_table(m, b, C[b]);
    int32_t *queue = (int32_t *)malloc((size_t)(N > 0 ? N : 1) * sizeof(int32_t));
    if (!queue) return -1;
    int status = 0;
    int64_t nr = *n_rast;
    for (int64_t t = t0; t < t0 + n_steps; ++t) {
        const int64_t slot = t % OR_DMAX;
        int64_t nq = 0;
        int b = 0;
        for (int64_t i = 0; i < N; ++i) {
            while (i >= pop_off[b + 1]) ++b;
            const int32_t T = or_poisson_count(or_poisson_uniform(seed, t, i), C[b]);
            const double in = W[slot * N + i] + (double)T * w_ext;
            W[slot * N + i] = 0.0;
            int spike = 0;
            if (R[i] == 0) {
                double x = p22 * U[i] + p21 * I[i];
                if (x >= theta) {
                    spike = 1;
                    x = u_reset;
                    R[i] = t_ref;
                }
                U[i] = x;
            } else {
                U[i] = u_reset;
                R[i] -= 1;
            }
            I[i] = p11 * I[i] + in;
            if (spike) {
                queue[nq++] = (int32_t)i;
                if (nr < rast_cap) {
                    rast_t[nr] = (int32_t)t;
                    rast_i[nr] = (int32_t)i;
                } else if (status == 0) {
                    status = 1;
                }
                ++nr;
            }
        }
        for (int64_t q = 0; q < nq; ++q) {
            const int64_t s = queue[q];
            for (int64_t e = row_ptr[s]; e < row_ptr[s + 1]; ++e) W[((t + dly[e]) % OR_DMAX) * N + post[e]] += w_pA[e];
        }
    }
    *n_rast = nr;
    free(queue);
    return status;
}
