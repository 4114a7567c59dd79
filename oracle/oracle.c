/*
 * FP64 CPU oracle of the frequency-domain coherent beamformer.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the tests, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py load it.  It shares no code with the CUDA path.
 *
 * Every function is the plain definition, in double precision, with no
 * blocking, fusion or reordering beyond what the definition states:
 *
 *   weights   W[c][b][n] = exp(-i 2 pi f_c (r_n . s_b) / c0)        (Eq. 1;
 *             the phase that undoes a plane wave from s_b, Section 1), zero
 *             for masked-out antennas (antenna mask, Section 3.1)
 *   beams     B[b][c][t] = sum_n W[c][b][n] X[c][t][n]                (the
 *             per-channel matrix-vector product of Section 2.1)
 *   power     P[b][c][j] = sum_{t = j T_int}^{(j+1) T_int - 1} |B[b][c][t]|^2
 *             (power detection computed inside the beamformer, Section 2.1;
 *             non-overlapping windows from t = 0, a partial last window is
 *             dropped)
 *   incoherent P_inc[c][j] = sum_{t in window j} sum_n |X[c][t][n]|^2
 *             (square, then add: Section 1)
 *
 * Complex numbers are stored as interleaved (re, im) doubles.  Channels are
 * independent, so the only parallelism is one thread per channel range.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

static const double ORACLE_C0 = 299792458.0;   /* m/s, exact */
static const double ORACLE_PI = 3.14159265358979323846264338327950288;

int oracle_weights(int n_ant, const double *pos, const unsigned char *mask,
                   int n_chan, const double *freqs, int n_beam,
                   const double *dirs, double *w)
{
    if (n_ant <= 0 || n_chan <= 0 || n_beam <= 0) return 1;
    for (int c = 0; c < n_chan; ++c)
        for (int b = 0; b < n_beam; ++b)
            for (int n = 0; n < n_ant; ++n) {
                double *o = w + 2 * (((size_t)c * n_beam + b) * n_ant + n);
                if (mask && !mask[n]) { o[0] = 0.0; o[1] = 0.0; continue; }
                double rs = pos[3 * n] * dirs[3 * b] + pos[3 * n + 1] * dirs[3 * b + 1]
                          + pos[3 * n + 2] * dirs[3 * b + 2];
                double phase = 2.0 * ORACLE_PI * freqs[c] * rs / ORACLE_C0;
                o[0] = cos(phase);      /* exp(-i phase) */
                o[1] = -sin(phase);
            }
    return 0;
}

typedef struct {
    int n_ant, n_chan, n_samp, n_beam, t_int;
    const double *w, *x;
    double *out;
    int c0, c1;
    int nct;      /* 1: x is antenna-major [n][c][t][2] */
} job_t;

static const double *x_at(const job_t *j, int c, int t, int n)
{
    if (j->nct)
        return j->x + 2 * (((size_t)n * j->n_chan + c) * j->n_samp + t);
    return j->x + 2 * (((size_t)c * j->n_samp + t) * j->n_ant + n);
}

/* B[b][c][t] for one channel and beam */
static void beam_value(const job_t *j, int c, int b, int t, double *re, double *im)
{
    double sr = 0.0, si = 0.0;
    const double *wr = j->w + 2 * (((size_t)c * j->n_beam + b) * j->n_ant);
    for (int n = 0; n < j->n_ant; ++n) {
        const double *xv = x_at(j, c, t, n);
        double a = wr[2 * n], bb = wr[2 * n + 1];
        sr += a * xv[0] - bb * xv[1];
        si += a * xv[1] + bb * xv[0];
    }
    *re = sr;
    *im = si;
}

static void *beams_worker(void *arg)
{
    const job_t *j = (const job_t *)arg;
    for (int c = j->c0; c < j->c1; ++c)
        for (int b = 0; b < j->n_beam; ++b)
            for (int t = 0; t < j->n_samp; ++t) {
                double *o = j->out + 2 * (((size_t)b * j->n_chan + c) * j->n_samp + t);
                beam_value(j, c, b, t, &o[0], &o[1]);
            }
    return NULL;
}

static void *power_worker(void *arg)
{
    const job_t *j = (const job_t *)arg;
    int n_out = j->n_samp / j->t_int;
    for (int c = j->c0; c < j->c1; ++c)
        for (int b = 0; b < j->n_beam; ++b)
            for (int q = 0; q < n_out; ++q) {
                double acc = 0.0;
                for (int t = q * j->t_int; t < (q + 1) * j->t_int; ++t) {
                    double re, im;
                    beam_value(j, c, b, t, &re, &im);
                    acc += re * re + im * im;
                }
                j->out[((size_t)b * j->n_chan + c) * n_out + q] = acc;
            }
    return NULL;
}

static void *incoherent_worker(void *arg)
{
    const job_t *j = (const job_t *)arg;
    int n_out = j->n_samp / j->t_int;
    for (int c = j->c0; c < j->c1; ++c)
        for (int q = 0; q < n_out; ++q) {
            double acc = 0.0;
            for (int t = q * j->t_int; t < (q + 1) * j->t_int; ++t)
                for (int n = 0; n < j->n_ant; ++n) {
                    const double *xv = x_at(j, c, t, n);
                    acc += xv[0] * xv[0] + xv[1] * xv[1];
                }
            j->out[(size_t)c * n_out + q] = acc;
        }
    return NULL;
}

static int run_threads(job_t base, int n_threads, void *(*fn)(void *))
{
    if (n_threads <= 0) n_threads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > base.n_chan) n_threads = base.n_chan;
    pthread_t *tid = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    job_t *jobs = (job_t *)calloc((size_t)n_threads, sizeof(job_t));
    if (!tid || !jobs) { free(tid); free(jobs); return 2; }
    for (int i = 0; i < n_threads; ++i) {
        jobs[i] = base;
        jobs[i].c0 = (int)((long)base.n_chan * i / n_threads);
        jobs[i].c1 = (int)((long)base.n_chan * (i + 1) / n_threads);
        pthread_create(&tid[i], NULL, fn, &jobs[i]);
    }
    for (int i = 0; i < n_threads; ++i) pthread_join(tid[i], NULL);
    free(tid);
    free(jobs);
    return 0;
}

/* beams[b][c][t][2]; x layout: nct = 0 -> [c][t][n][2], 1 -> [n][c][t][2] */
int oracle_beams(int n_ant, int n_chan, int n_samp, int n_beam, const double *w,
                 const double *x, int nct, double *beams, int n_threads)
{
    if (n_ant <= 0 || n_chan <= 0 || n_samp < 0 || n_beam <= 0) return 1;
    job_t j = {n_ant, n_chan, n_samp, n_beam, 1, w, x, beams, 0, 0, nct};
    return run_threads(j, n_threads, beams_worker);
}

/* power[b][c][n_samp / t_int] */
int oracle_power(int n_ant, int n_chan, int n_samp, int n_beam, const double *w,
                 const double *x, int nct, int t_int, double *power, int n_threads)
{
    if (n_ant <= 0 || n_chan <= 0 || n_samp < 0 || n_beam <= 0 || t_int <= 0) return 1;
    job_t j = {n_ant, n_chan, n_samp, n_beam, t_int, w, x, power, 0, 0, nct};
    return run_threads(j, n_threads, power_worker);
}

/* power[c][n_samp / t_int] */
int oracle_incoherent(int n_ant, int n_chan, int n_samp, const double *x, int nct,
                      int t_int, double *power, int n_threads)
{
    if (n_ant <= 0 || n_chan <= 0 || n_samp < 0 || t_int <= 0) return 1;
    job_t j = {n_ant, n_chan, n_samp, 1, t_int, NULL, x, power, 0, 0, nct};
    return run_threads(j, n_threads, incoherent_worker);
}
