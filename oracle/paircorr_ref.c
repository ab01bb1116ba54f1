/*
 * FP64 CPU oracle for the space- and time-displaced spin pair correlation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * What it computes (arXiv 2308.07487):
 *   Eq. 4   C^a(r-r',t) = <S^a_r(t) S^a_r'(0)> - <S^a_r(t)><S^a_r'(0)>
 *   Eq. 5   the same quantity as the average of centred products
 *   Eq. 3   S(q,t) = (1/N) sum_a sum_{r,r'} e^{-i q.(r-r')} C^a(r-r',t)  (real part)
 *   Eq. 6   Q(i,j) = e^{-i q.(r_i - r_j)}
 * The statistical average <.> runs over time origins t0 = 0..T0-1 and over the
 * S samples that are concatenated along the contraction axis (the paper averages
 * over M Monte Carlo realisations at one origin, Section 3.1: that is the case
 * T0 = 1, S = M).  As in Algorithm 2, every (r, r') pair is visited by a plain
 * loop with the realisation/origin sum innermost and the three components
 * handled together (Section 3.1, first optimisation).
 *
 * Binned form.  For each displacement t in t_list and each distance bin b:
 *   C_sum[t][b] = sum over ordered pairs (i,j), i == j included, with bin(i,j) == b, of
 *                 G_ij(t) = sum_{s,t0,a} A_{i,s,a}(t0+t) * B_{j,s,a}(t0)
 *   M_abs[t][b] = sum over the same pairs of |G_ij(t)|   (scale of the bin, for errors)
 *   P_abs[t][b] = sum over the same pairs of sum_{s,t0,a} |A * B|  (the scale of any
 *                 rounding-error bound of the sum: |fl(G) - G| <= c u sum |A B|)
 *   counts[b]   = number of such ordered pairs
 * A = B = S (center = 0), or both centred by their origin/sample means (center = 1,
 * Eq. 5).  The normalised correlation is C(b,t) = C_sum / (S*T0*counts).
 * Phase form:  Sq_sum[t][q] = sum_{i,j} cos(q.(r_i - r_j)) G_ij(t);
 *              S(q,t) = Sq_sum / (N*S*T0).
 *              Sq_abs[t][q] = sum_{i,j} |cos(q.(r_i - r_j)) G_ij(t)|  (scale of that q's
 *              sum, for errors: the phase-form counterpart of M_abs)
 * Sine part:   Sq_im[t][q]  = sum_{i,j} sin(q.(r_i - r_j)) G_ij(t)  (Eq. 3's imaginary
 *              part of e^{-iq.(r_i - r_j)} is minus this); Sq_im_abs likewise.
 *
 * Distance bins.  bin(i,j) = max{k >= 0 : (k*w)^2 <= d2(i,j)}, dropped if >= n_bins.
 *   lattice geometry:   d2 = exact integer squared displacement of the integer
 *                       coordinates, minimum image per axis when periodic.
 *   position geometry:  d2 = FP32 value of  fmaf(dz,dz, fmaf(dy,dy, dx*dx)) with
 *                       dx = x_j - x_i etc. computed in FP32 (no contraction).
 * Build with -ffp-contract=off so the FP32 rule is evaluated exactly as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* smallest k >= 0 with ((k+1) w)^2 > d2, i.e. the largest k with (k w)^2 <= d2 */
static int64_t bin_of_d2(double d2, double w)
{
    int64_t k = (int64_t)floor(sqrt(d2) / w);
    if (k < 0) k = 0;
    while (k > 0 && (k * w) * (k * w) > d2) --k;
    while (((k + 1) * w) * ((k + 1) * w) <= d2) ++k;
    return k;
}

static int64_t min_image(int64_t d, int64_t L, int periodic)
{
    if (d < 0) d = -d;
    if (periodic && L - d < d) d = L - d;
    return d;
}

/* squared distance of pair (i,j) under the geometry rules above */
static double pair_d2(int geom, int64_t i, int64_t j, const int32_t *coords,
                      const int32_t *L, int periodic, const float *pos)
{
    if (geom == 0) {
        int64_t s = 0;
        for (int a = 0; a < 3; ++a) {
            int64_t d = min_image((int64_t)coords[3 * j + a] - coords[3 * i + a], L[a], periodic);
            s += d * d;
        }
        return (double)s;
    } else {
        float dx = pos[3 * j + 0] - pos[3 * i + 0];
        float dy = pos[3 * j + 1] - pos[3 * i + 1];
        float dz = pos[3 * j + 2] - pos[3 * i + 2];
        float xx = dx * dx;
        float d2 = fmaf(dz, dz, fmaf(dy, dy, xx));
        return (double)d2;
    }
}

int oracle_bin_of_d2(double d2, double w) { return (int)bin_of_d2(d2, w); }

/* Threads of the next parallel loop (OMP_NUM_THREADS, else the CPUs this process may
 * run on): the core count a timing of the oracle reports. */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sets the threads of the following parallel loops (n >= 1). */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

double oracle_pair_d2(int geom, int64_t i, int64_t j, const int32_t *coords,
                      const int32_t *L, int periodic, const float *pos)
{
    return pair_d2(geom, i, j, coords, L, periodic, pos);
}

/* Ordered-pair counts per bin over rows [row_begin,row_end) x all columns. */
int oracle_pair_counts(int64_t N, int geom, const int32_t *coords, const int32_t *L,
                       int periodic, const float *pos, double w, int64_t n_bins,
                       int64_t row_begin, int64_t row_end, int64_t *counts)
{
    memset(counts, 0, sizeof(int64_t) * (size_t)n_bins);
#pragma omp parallel
    {
        int64_t *loc = (int64_t *)calloc((size_t)n_bins, sizeof(int64_t));
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = row_begin; i < row_end; ++i)
            for (int64_t j = 0; j < N; ++j) {
                int64_t b = bin_of_d2(pair_d2(geom, i, j, coords, L, periodic, pos), w);
                if (b < n_bins) loc[b] += 1;
            }
#pragma omp critical
        for (int64_t b = 0; b < n_bins; ++b) counts[b] += loc[b];
        free(loc);
    }
    return 0;
}

/*
 * traj: [N][S][F][3] FP32.  t_list: n_tl displacements, each with t + T0 <= F.
 * Outputs (caller-allocated, overwritten): C_sum, M_abs [n_tl][n_bins];
 * Sq_sum, Sq_im, Sq_abs, Sq_im_abs [n_tl][n_q] (may be NULL); counts [n_bins] (may be NULL).
 * q: [n_q][3] FP64.  Phase positions are the integer coordinates (geom 0) or pos.
 */
int oracle_pair_corr(int64_t N, int64_t F, int64_t S, int64_t T0,
                     int64_t n_tl, const int32_t *t_list, const float *traj,
                     int geom, const int32_t *coords, const int32_t *L, int periodic,
                     const float *pos, double w, int64_t n_bins,
                     int64_t n_q, const double *q, int center,
                     int64_t row_begin, int64_t row_end,
                     double *C_sum, double *M_abs, double *P_abs, double *Sq_sum,
                     double *Sq_im, double *Sq_abs, double *Sq_im_abs, int64_t *counts)
{
    if (row_begin < 0 || row_end > N || row_begin > row_end) return -1;
    for (int64_t k = 0; k < n_tl; ++k)
        if (t_list[k] < 0 || t_list[k] + T0 > F) return -2;

    const int64_t nc = n_tl * n_bins, nq = n_tl * n_q;
    memset(C_sum, 0, sizeof(double) * (size_t)nc);
    memset(M_abs, 0, sizeof(double) * (size_t)nc);
    if (P_abs) memset(P_abs, 0, sizeof(double) * (size_t)nc);
    if (Sq_sum) memset(Sq_sum, 0, sizeof(double) * (size_t)nq);
    if (Sq_im) memset(Sq_im, 0, sizeof(double) * (size_t)nq);
    if (Sq_abs) memset(Sq_abs, 0, sizeof(double) * (size_t)nq);
    if (Sq_im_abs) memset(Sq_im_abs, 0, sizeof(double) * (size_t)nq);
    if (counts) memset(counts, 0, sizeof(int64_t) * (size_t)n_bins);

#define TR(i, s, f, a) ((double)traj[(((i) * S + (s)) * F + (f)) * 3 + (a)])

    /* Eq. 5 means: mB[j][a] over (s, t0 < T0); mA[i][k][a] over (s, t0+t_k). */
    double *mB = NULL, *mA = NULL;
    if (center) {
        mB = (double *)calloc((size_t)(N * 3), sizeof(double));
        mA = (double *)calloc((size_t)(N * n_tl * 3), sizeof(double));
        for (int64_t i = 0; i < N; ++i)
            for (int64_t s = 0; s < S; ++s)
                for (int64_t t0 = 0; t0 < T0; ++t0)
                    for (int a = 0; a < 3; ++a) {
                        mB[3 * i + a] += TR(i, s, t0, a) / (double)(S * T0);
                        for (int64_t k = 0; k < n_tl; ++k)
                            mA[(i * n_tl + k) * 3 + a] += TR(i, s, t0 + t_list[k], a) / (double)(S * T0);
                    }
    }

    int err = 0;
#pragma omp parallel
    {
        double *c_loc = (double *)calloc((size_t)nc, sizeof(double));
        double *m_loc = (double *)calloc((size_t)nc, sizeof(double));
        double *p_loc = (double *)calloc((size_t)nc, sizeof(double));
        double *q_loc = (double *)calloc((size_t)(nq > 0 ? nq : 1), sizeof(double));
        double *qs_loc = (double *)calloc((size_t)(nq > 0 ? nq : 1), sizeof(double));
        double *qa_loc = (double *)calloc((size_t)(nq > 0 ? nq : 1), sizeof(double));
        double *qsa_loc = (double *)calloc((size_t)(nq > 0 ? nq : 1), sizeof(double));
        int64_t *n_loc = (int64_t *)calloc((size_t)n_bins, sizeof(int64_t));
        double *ph = (double *)calloc((size_t)(n_q > 0 ? n_q : 1), sizeof(double));
        double *phs = (double *)calloc((size_t)(n_q > 0 ? n_q : 1), sizeof(double));
        if (!c_loc || !m_loc || !p_loc || !q_loc || !qs_loc || !qa_loc || !qsa_loc || !n_loc ||
            !ph || !phs)
            err = 1;
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = row_begin; i < row_end; ++i) {
            if (err) continue;
            for (int64_t j = 0; j < N; ++j) {
                int64_t b = bin_of_d2(pair_d2(geom, i, j, coords, L, periodic, pos), w);
                int binned = b < n_bins;
                if (!binned && n_q == 0) continue;
                if (binned) n_loc[b] += 1;
                for (int64_t iq = 0; iq < n_q; ++iq) {
                    double arg = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        double ri = geom == 0 ? (double)coords[3 * i + a] : (double)pos[3 * i + a];
                        double rj = geom == 0 ? (double)coords[3 * j + a] : (double)pos[3 * j + a];
                        arg += q[3 * iq + a] * (ri - rj);
                    }
                    ph[iq] = cos(arg);
                    phs[iq] = sin(arg);
                }
                for (int64_t k = 0; k < n_tl; ++k) {
                    const int64_t t = t_list[k];
                    double g = 0.0, gabs = 0.0;
                    for (int64_t s = 0; s < S; ++s)
                        for (int64_t t0 = 0; t0 < T0; ++t0)
                            for (int a = 0; a < 3; ++a) {
                                double x = TR(i, s, t0 + t, a);
                                double y = TR(j, s, t0, a);
                                if (center) {
                                    x -= mA[(i * n_tl + k) * 3 + a];
                                    y -= mB[3 * j + a];
                                }
                                g += x * y;
                                gabs += fabs(x * y);
                            }
                    if (binned) {
                        c_loc[k * n_bins + b] += g;
                        m_loc[k * n_bins + b] += fabs(g);
                        p_loc[k * n_bins + b] += gabs;
                    }
                    for (int64_t iq = 0; iq < n_q; ++iq) {
                        q_loc[k * n_q + iq] += ph[iq] * g;
                        qs_loc[k * n_q + iq] += phs[iq] * g;
                        qa_loc[k * n_q + iq] += fabs(ph[iq] * g);
                        qsa_loc[k * n_q + iq] += fabs(phs[iq] * g);
                    }
                }
            }
        }
#pragma omp critical
        {
            if (c_loc && m_loc && p_loc && q_loc && qs_loc && qa_loc && qsa_loc && n_loc) {
                for (int64_t x = 0; x < nc; ++x) {
                    C_sum[x] += c_loc[x];
                    M_abs[x] += m_loc[x];
                    if (P_abs) P_abs[x] += p_loc[x];
                }
                if (Sq_sum) for (int64_t x = 0; x < nq; ++x) Sq_sum[x] += q_loc[x];
                if (Sq_im) for (int64_t x = 0; x < nq; ++x) Sq_im[x] += qs_loc[x];
                if (Sq_abs) for (int64_t x = 0; x < nq; ++x) Sq_abs[x] += qa_loc[x];
                if (Sq_im_abs) for (int64_t x = 0; x < nq; ++x) Sq_im_abs[x] += qsa_loc[x];
                if (counts) for (int64_t b = 0; b < n_bins; ++b) counts[b] += n_loc[b];
            }
        }
        free(c_loc); free(m_loc); free(p_loc); free(q_loc); free(qs_loc); free(qa_loc);
        free(qsa_loc); free(n_loc);
        free(ph); free(phs);
    }
#undef TR
    free(mA);
    free(mB);
    return err ? -3 : 0;
}

/*
 * Eq. 4 form (product average minus product of averages), for the Eq. 4 == Eq. 5
 * check: G4_ij(t) = sum_{s,t0,a} S_i(t0+t) S_j(t0) - S*T0 * mA_i(t) . mB_j.
 * Binned like oracle_pair_corr; lattice or position geometry.
 */
int oracle_pair_corr_eq4(int64_t N, int64_t F, int64_t S, int64_t T0,
                         int64_t n_tl, const int32_t *t_list, const float *traj,
                         int geom, const int32_t *coords, const int32_t *L, int periodic,
                         const float *pos, double w, int64_t n_bins, double *C_sum)
{
    memset(C_sum, 0, sizeof(double) * (size_t)(n_tl * n_bins));
#define TR(i, s, f, a) ((double)traj[(((i) * S + (s)) * F + (f)) * 3 + (a)])
    for (int64_t k = 0; k < n_tl; ++k) {
        const int64_t t = t_list[k];
        for (int64_t i = 0; i < N; ++i)
            for (int64_t j = 0; j < N; ++j) {
                int64_t b = bin_of_d2(pair_d2(geom, i, j, coords, L, periodic, pos), w);
                if (b >= n_bins) continue;
                double prod = 0.0, ma[3] = {0, 0, 0}, mb[3] = {0, 0, 0};
                for (int64_t s = 0; s < S; ++s)
                    for (int64_t t0 = 0; t0 < T0; ++t0)
                        for (int a = 0; a < 3; ++a) {
                            prod += TR(i, s, t0 + t, a) * TR(j, s, t0, a);
                            ma[a] += TR(i, s, t0 + t, a);
                            mb[a] += TR(j, s, t0, a);
                        }
                const double M = (double)(S * T0);
                double g = prod - (ma[0] * mb[0] + ma[1] * mb[1] + ma[2] * mb[2]) / M;
                C_sum[k * n_bins + b] += g;
            }
    }
#undef TR
    return 0;
}
