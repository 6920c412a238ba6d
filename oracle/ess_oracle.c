/*
 * ess_oracle.c -- plain FP64 CPU oracle for linear elliptical slice sampling
 * of linearly truncated normals (Wu & Gardner, arXiv 2407.10449).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA library is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never calls it, and it shares no code, header, table or helper
 * with the CUDA library.
 *
 * Everything is IEEE double precision, written step by step in the paper's
 * order and notation:
 *   - Alg. 1 (the chain):          draw nu ~ N(0, I), build the ellipse
 *                                   x cos(theta) + nu sin(theta), compute the
 *                                   active intervals, draw theta uniformly,
 *                                   move.
 *   - App. B (roots):              p = a.x, q = a.nu, r = sqrt(p^2 + q^2),
 *                                   tau = atan2(q, p), theta = tau +- arccos(b/r).
 *   - Sec. 3.2 (edge cases):       b/r > 1 -> no root (row ignored); b/r = 1
 *                                   treated the same; b/r = -1 -> alpha = 0,
 *                                   beta = 2 pi.
 *   - Alg. 2 (brute force):        I_act built by intersecting [0, 2 pi] with
 *                                   every I_i = [0, alpha_i] U [beta_i, 2 pi]
 *                                   in turn (pairwise clipping, O(m^2) worst).
 *   - Sec. 3.3 (robustness):       optional trimming of constraint endpoints
 *                                   by eps; rejection of an infeasible x_{t+1}.
 *   - App. A (whitening):          A' = A L, b' = b - A mu; x = L u + mu.
 *   - App. A (the factor L):       Sigma = L L^T by the Cholesky-Banachiewicz
 *                                   recurrence, row by row.
 *
 * Readings taken where the paper is silent (each one is also listed in the
 * design notes of the repository):
 *   - Wrapping (Sec. 2 only says "add or subtract a multiple of 2 pi"): tau is
 *     shifted into [0, 2 pi) and alpha = max(0, tau - h), beta = min(2 pi,
 *     tau + h).  For a feasible x the open infeasible arc never contains 0,
 *     so the clamps only absorb rounding.
 *   - r = 0 is treated as "no root" (App. B: a tautology when b >= 0).
 *   - b/r >= 1 is "no root" (Sec. 3.2 leaves b/r = 1 unhandled; the excluded
 *     set differs by one point).  b/r < -1 from rounding is clamped to -1.
 *   - theta ~ U(I_act) (Alg. 1 line "sample uniformly") is drawn by the
 *     inverse CDF over the pieces in ascending order: s = u L, theta =
 *     l_j + (s - S_{j-1}) for the first piece j with s < S_j.  If L = 0,
 *     theta = 0 (the chain stays at x_t).
 *   - Trimming (Sec. 3.3, eps not given): only endpoints that are constraint
 *     angles move; the glued point 0 / 2 pi never does.  A piece whose ends
 *     cross is dropped.
 *   - Rejection (Sec. 3.3): x_{t+1} is rejected iff max_i (a_i.x_{t+1} - b_i)
 *     > 0 in double precision, with no slack.
 *
 * Random numbers (not from the paper, which does not say how nu is drawn):
 * Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) keyed by the 64-bit seed,
 * counter (block n, chain, iteration t, (problem << 8) | stream), and the
 * Box-Muller transform:
 *   u1 = (r0 + 1) / 2^32 in (0, 1], u2 = r1 / 2^32 in [0, 1),
 *   z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = sqrt(-2 ln u1) sin(2 pi u2);
 * the same for (r2, r3) -> z2, z3.  nu_j uses block n = j / 4, output j % 4,
 * stream 0.  The uniform for theta uses block 0 of stream 1:
 *   u = ((r0 >> 5) * 2^26 + (r1 >> 6)) / 2^53 in [0, 1).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TWO_PI (2.0 * M_PI)

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 from its published definition.                               */
/* ------------------------------------------------------------------------ */

static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u; /* golden ratio */
static const uint32_t PHILOX_W1 = 0xBB67AE85u; /* sqrt(3) - 1 */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One Philox block for (seed, n, chain, t, problem, stream). */
void orc_rng_block(uint64_t seed, uint32_t n, uint32_t chain, uint32_t t,
                   uint32_t problem, uint32_t stream, uint32_t out[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {n, chain, t, (problem << 8) | (stream & 0xFFu)};
    orc_philox4x32_10(ctr, key, out);
}

/* nu ~ N(0, I_d) for one chain at iteration t (Alg. 1: "sample nu_t"). */
void orc_draw_nu(uint64_t seed, uint32_t chain, uint32_t t, uint32_t problem,
                 int d, double *nu)
{
    const double two32 = 4294967296.0;
    for (int n = 0; 4 * n < d; ++n) {
        uint32_t r[4];
        orc_rng_block(seed, (uint32_t)n, chain, t, problem, 0u, r);
        double z[4];
        for (int pair = 0; pair < 2; ++pair) {
            double u1 = ((double)r[2 * pair] + 1.0) / two32;   /* (0, 1] */
            double u2 = (double)r[2 * pair + 1] / two32;       /* [0, 1) */
            double radius = sqrt(-2.0 * log(u1));
            z[2 * pair] = radius * cos(ORC_TWO_PI * u2);
            z[2 * pair + 1] = radius * sin(ORC_TWO_PI * u2);
        }
        for (int k = 0; k < 4 && 4 * n + k < d; ++k) nu[4 * n + k] = z[k];
    }
}

/* u ~ U[0, 1) with 53 random bits for the theta draw (stream 1). */
double orc_draw_u(uint64_t seed, uint32_t chain, uint32_t t, uint32_t problem)
{
    uint32_t r[4];
    orc_rng_block(seed, 0u, chain, t, problem, 1u, r);
    uint64_t hi = (uint64_t)(r[0] >> 5);  /* 27 bits */
    uint64_t lo = (uint64_t)(r[1] >> 6);  /* 26 bits */
    return (double)(hi * 67108864ull + lo) / 9007199254740992.0; /* / 2^53 */
}

/* ------------------------------------------------------------------------ */
/* Roots of a.x cos(theta) + a.nu sin(theta) = b   (App. B, Sec. 3.2).        */
/* ------------------------------------------------------------------------ */

/* Returns 1 and the open infeasible arc (alpha, beta) if the equation has two
 * roots (or the b/r = -1 single root), 0 if the constraint can be ignored
 * (b/r >= 1 or r = 0).  Returns -1 if the data prove x infeasible (r = 0 and
 * b < 0). */
int orc_roots(double p, double q, double b, double *alpha, double *beta)
{
    double r = sqrt(p * p + q * q);
    if (r == 0.0) {
        *alpha = 0.0; *beta = 0.0;
        return b >= 0.0 ? 0 : -1;
    }
    double ratio = b / r;
    if (ratio >= 1.0) {           /* no intersection, or tangent from inside */
        *alpha = 0.0; *beta = 0.0;
        return 0;
    }
    if (ratio < -1.0) ratio = -1.0;  /* x on the hyperplane, rounding */
    double tau = atan2(q, p);        /* cos tau = p / r, sin tau = q / r */
    if (tau < 0.0) tau += ORC_TWO_PI;
    double h = acos(ratio);          /* cos(theta - tau) = b / r */
    double lo = tau - h, hi = tau + h;
    *alpha = lo > 0.0 ? lo : 0.0;
    *beta = hi < ORC_TWO_PI ? hi : ORC_TWO_PI;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2: I_act = intersection of the I_i, by sequential clipping.           */
/* ------------------------------------------------------------------------ */

typedef struct {
    double lo, hi;
    int lo_is_root, hi_is_root;   /* endpoint is a constraint angle (for trim) */
} orc_piece;

/* Intersects [0, 2 pi] with [0, alpha_i] U [beta_i, 2 pi] for every row with
 * use[i] != 0 (or every row if use == NULL).  Writes the pieces in ascending
 * order; returns their count, or -1 if cap is too small.  Zero-length pieces
 * (lo == hi) are kept: they are part of the set. */
static int orc_clip_all(int m, const double *alpha, const double *beta,
                        const int *use, orc_piece *out, int cap)
{
    orc_piece *cur = (orc_piece *)malloc(sizeof(orc_piece) * (size_t)(m + 2) * 2);
    orc_piece *nxt = (orc_piece *)malloc(sizeof(orc_piece) * (size_t)(m + 2) * 2);
    int n = 1;
    cur[0].lo = 0.0; cur[0].hi = ORC_TWO_PI;
    cur[0].lo_is_root = 0; cur[0].hi_is_root = 0;
    for (int i = 0; i < m; ++i) {
        if (use && !use[i]) continue;
        int k = 0;
        for (int j = 0; j < n; ++j) {
            orc_piece s = cur[j];
            /* s intersect [0, alpha_i] */
            orc_piece left = s;
            if (alpha[i] < s.hi) { left.hi = alpha[i]; left.hi_is_root = 1; }
            if (left.lo <= left.hi) nxt[k++] = left;
            /* s intersect [beta_i, 2 pi] */
            orc_piece right = s;
            if (beta[i] > s.lo) { right.lo = beta[i]; right.lo_is_root = 1; }
            if (right.lo <= right.hi) {
                /* a zero-measure overlap with `left' (alpha_i == beta_i cannot
                 * happen for a row with roots, but s may be a single point) */
                if (!(k > 0 && nxt[k - 1].lo == right.lo && nxt[k - 1].hi == right.hi))
                    nxt[k++] = right;
            }
        }
        orc_piece *tmp = cur; cur = nxt; nxt = tmp;
        n = k;
    }
    int ret = n;
    if (n > cap) ret = -1;
    else memcpy(out, cur, sizeof(orc_piece) * (size_t)n);
    free(cur); free(nxt);
    return ret;
}

/* Public form of Alg. 2 on given (alpha, beta) pairs.  lo/hi get the pieces
 * in ascending order (zero-length pieces included).  Returns the number of
 * pieces or -1 if cap is too small. */
int orc_active_intervals(int m, const double *alpha, const double *beta,
                         const int *use, double *lo, double *hi, int cap)
{
    orc_piece *buf = (orc_piece *)malloc(sizeof(orc_piece) * (size_t)(m + 2) * 2);
    int n = orc_clip_all(m, alpha, beta, use, buf, (m + 2) * 2);
    if (n >= 0 && n <= cap) {
        for (int j = 0; j < n; ++j) { lo[j] = buf[j].lo; hi[j] = buf[j].hi; }
    } else {
        n = -1;
    }
    free(buf);
    return n;
}

/* Sec. 3.3 trimming: constraint endpoints move inwards by eps; 0 and 2 pi do
 * not move; a piece whose ends cross is dropped.  Returns the new count. */
static int orc_trim(orc_piece *pc, int n, double eps)
{
    if (eps <= 0.0) return n;
    int k = 0;
    for (int j = 0; j < n; ++j) {
        orc_piece s = pc[j];
        if (s.lo_is_root) s.lo += eps;
        if (s.hi_is_root) s.hi -= eps;
        if (s.lo <= s.hi) pc[k++] = s;
    }
    return k;
}

/* theta ~ U(I_act) by the inverse CDF over ascending pieces. */
double orc_draw_theta(int n, const double *lo, const double *hi, double u)
{
    double total = 0.0;
    for (int j = 0; j < n; ++j) total += hi[j] - lo[j];
    if (!(total > 0.0)) return 0.0;
    double s = u * total;
    double cum = 0.0;
    int last = -1;
    for (int j = 0; j < n; ++j) {
        double len = hi[j] - lo[j];
        if (len > 0.0) last = j;
        if (s < cum + len) {
            double theta = lo[j] + (s - cum);
            return theta < hi[j] ? theta : hi[j];
        }
        cum += len;
    }
    return last >= 0 ? hi[last] : 0.0;
}

/* ------------------------------------------------------------------------ */
/* One chain step with given draws (Alg. 1 body + Sec. 3.3).                  */
/* ------------------------------------------------------------------------ */

/* a_i . v for row i of the row-major m x d matrix A. */
static double orc_row_dot(const double *A, int d, int i, const double *v)
{
    const double *a = A + (size_t)i * (size_t)d;
    double s = 0.0;
    for (int j = 0; j < d; ++j) s += a[j] * v[j];
    return s;
}

/* Maximum residual max_i (a_i . x - b_i). */
double orc_max_residual(const double *A, const double *b, int d, int m, const double *x)
{
    double worst = -INFINITY;
    for (int i = 0; i < m; ++i) {
        double r = orc_row_dot(A, d, i, x) - b[i];
        if (r > worst) worst = r;
    }
    return worst;
}

/* status codes of orc_step */
#define ORC_OK 0
#define ORC_INFEASIBLE_X (-1)
#define ORC_CAP (-2)

/*
 * x_next = x cos(theta) + nu sin(theta) with theta ~ U(I_act) drawn from u.
 * Outputs (any may be NULL): the active pieces (after trimming) in lo/hi with
 * their count in *n_pieces (cap entries at most), theta, whether the move was
 * rejected, and the per-row roots alpha/beta/has_root (m entries each).
 */
int orc_step(const double *A, const double *b, int d, int m,
             const double *x, const double *nu, double u, double trim_eps,
             double *x_next, double *lo, double *hi, int cap, int *n_pieces,
             double *theta_out, int *rejected,
             double *alpha_out, double *beta_out, int *has_root_out)
{
    double *alpha = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *beta = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    int *use = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    orc_piece *pc = (orc_piece *)malloc(sizeof(orc_piece) * (size_t)(m + 2) * 2);
    int status = ORC_OK;

    for (int i = 0; i < m; ++i) {
        double p = orc_row_dot(A, d, i, x);   /* App. B: p = a_i . x */
        double q = orc_row_dot(A, d, i, nu);  /*         q = a_i . nu */
        int k = orc_roots(p, q, b[i], &alpha[i], &beta[i]);
        if (k < 0 || p > b[i]) status = ORC_INFEASIBLE_X;  /* Alg. 1 needs x in D */
        use[i] = k > 0;
        if (alpha_out) alpha_out[i] = alpha[i];
        if (beta_out) beta_out[i] = beta[i];
        if (has_root_out) has_root_out[i] = use[i];
    }
    int n = orc_clip_all(m, alpha, beta, use, pc, (m + 2) * 2);
    n = orc_trim(pc, n, trim_eps);

    double *plo = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *phi = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int j = 0; j < n; ++j) { plo[j] = pc[j].lo; phi[j] = pc[j].hi; }
    double theta = orc_draw_theta(n, plo, phi, u);

    double c = cos(theta), s = sin(theta);
    for (int j = 0; j < d; ++j) x_next[j] = x[j] * c + nu[j] * s;
    int rej = 0;
    if (m > 0 && orc_max_residual(A, b, d, m, x_next) > 0.0) {
        rej = 1;                                   /* Sec. 3.3: stay at x_t */
        memcpy(x_next, x, sizeof(double) * (size_t)d);
    }

    if (n_pieces) *n_pieces = n;
    if (lo && hi) {
        if (n > cap) status = status ? status : ORC_CAP;
        for (int j = 0; j < n && j < cap; ++j) { lo[j] = plo[j]; hi[j] = phi[j]; }
    }
    if (theta_out) *theta_out = theta;
    if (rejected) *rejected = rej;

    free(plo); free(phi); free(pc); free(use); free(beta); free(alpha);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Many independent chains (Alg. 1 loop), threaded over chains.               */
/* ------------------------------------------------------------------------ */

typedef struct {
    const double *A, *b;
    int d, m;
    double *X;                 /* n_chains x d, updated in place */
    int chain_begin, chain_end;
    uint32_t chain_offset;     /* global chain id of row 0 */
    uint32_t t0;
    int n_iter;
    uint64_t seed;
    uint32_t problem;
    double trim_eps;
    double *samples;           /* optional: n_chains x n_rec x d */
    int record_every, n_rec;
    long long *rejections;     /* per chain */
    int status;
} orc_run_job;

static void *orc_run_worker(void *arg)
{
    orc_run_job *job = (orc_run_job *)arg;
    int d = job->d, m = job->m;
    double *nu = (double *)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
    double *xn = (double *)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
    for (int c = job->chain_begin; c < job->chain_end; ++c) {
        double *x = job->X + (size_t)c * (size_t)d;
        long long rej_count = 0;
        uint32_t gchain = job->chain_offset + (uint32_t)c;
        for (int it = 0; it < job->n_iter; ++it) {
            uint32_t t = job->t0 + (uint32_t)it;
            orc_draw_nu(job->seed, gchain, t, job->problem, d, nu);
            double u = orc_draw_u(job->seed, gchain, t, job->problem);
            int rej = 0;
            int st = orc_step(job->A, job->b, d, m, x, nu, u, job->trim_eps, xn,
                              NULL, NULL, 0, NULL, NULL, &rej, NULL, NULL, NULL);
            if (st != ORC_OK) job->status = st;
            rej_count += rej;
            memcpy(x, xn, sizeof(double) * (size_t)d);
            if (job->samples && job->record_every > 0 && (it + 1) % job->record_every == 0) {
                int k = (it + 1) / job->record_every - 1;
                if (k < job->n_rec)
                    memcpy(job->samples + ((size_t)c * (size_t)job->n_rec + (size_t)k) * (size_t)d,
                           x, sizeof(double) * (size_t)d);
            }
        }
        if (job->rejections) job->rejections[c] += rej_count;
    }
    free(xn); free(nu);
    return NULL;
}

/*
 * Runs n_chains independent chains for n_iter iterations starting at
 * iteration index t0.  X (n_chains x d) holds the start points and receives
 * the final states.  If samples != NULL, the state after every record_every-th
 * iteration is stored (n_chains x (n_iter / record_every) x d).  rejections
 * (n_chains, may be NULL) is incremented.  Returns ORC_OK or the first error.
 */
int orc_run(const double *A, const double *b, int d, int m,
            double *X, int n_chains, uint32_t chain_offset, uint32_t t0, int n_iter,
            uint64_t seed, uint32_t problem, double trim_eps,
            double *samples, int record_every, long long *rejections, int n_threads)
{
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_chains) n_threads = n_chains > 0 ? n_chains : 1;
    /* x_0 must lie in D (Alg. 1, first line) */
    for (int c = 0; c < n_chains; ++c)
        if (m > 0 && orc_max_residual(A, b, d, m, X + (size_t)c * (size_t)d) > 0.0)
            return ORC_INFEASIBLE_X;
    int n_rec = record_every > 0 ? n_iter / record_every : 0;
    orc_run_job *jobs = (orc_run_job *)calloc((size_t)n_threads, sizeof(orc_run_job));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int w = 0; w < n_threads; ++w) {
        orc_run_job *j = &jobs[w];
        j->A = A; j->b = b; j->d = d; j->m = m; j->X = X;
        j->chain_begin = (int)((long long)n_chains * w / n_threads);
        j->chain_end = (int)((long long)n_chains * (w + 1) / n_threads);
        j->chain_offset = chain_offset; j->t0 = t0; j->n_iter = n_iter;
        j->seed = seed; j->problem = problem; j->trim_eps = trim_eps;
        j->samples = samples; j->record_every = record_every; j->n_rec = n_rec;
        j->rejections = rejections; j->status = ORC_OK;
        pthread_create(&th[w], NULL, orc_run_worker, j);
    }
    int status = ORC_OK;
    for (int w = 0; w < n_threads; ++w) {
        pthread_join(th[w], NULL);
        if (jobs[w].status != ORC_OK && status == ORC_OK) status = jobs[w].status;
    }
    free(th); free(jobs);
    return status;
}

/* ------------------------------------------------------------------------ */
/* App. A: change of variables for N(mu, Sigma), Sigma = L L^T.              */
/* ------------------------------------------------------------------------ */

/* A_out = A L (m x d), b_out = b - A mu. */
void orc_whiten(const double *A, const double *b, const double *mu, const double *L,
                int d, int m, double *A_out, double *b_out)
{
    for (int i = 0; i < m; ++i) {
        const double *a = A + (size_t)i * (size_t)d;
        for (int k = 0; k < d; ++k) {
            double s = 0.0;
            for (int j = 0; j < d; ++j) s += a[j] * L[(size_t)j * (size_t)d + (size_t)k];
            A_out[(size_t)i * (size_t)d + (size_t)k] = s;
        }
        double am = 0.0;
        for (int j = 0; j < d; ++j) am += a[j] * (mu ? mu[j] : 0.0);
        b_out[i] = b[i] - am;
    }
}

/* X = U L^T + mu row by row: x = L u + mu for each of the n rows of U. */
void orc_unwhiten(const double *L, const double *mu, int d, int n, const double *U, double *X)
{
    for (int r = 0; r < n; ++r) {
        const double *u = U + (size_t)r * (size_t)d;
        double *x = X + (size_t)r * (size_t)d;
        for (int i = 0; i < d; ++i) {
            double s = 0.0;
            for (int j = 0; j < d; ++j) s += L[(size_t)i * (size_t)d + (size_t)j] * u[j];
            x[i] = s + (mu ? mu[i] : 0.0);
        }
    }
}

/* App. A needs a factor L with Sigma = L L^T.  Cholesky-Banachiewicz, row by
 * row: L_ij = (S_ij - sum_{k<j} L_ik L_jk) / L_jj for j < i, and
 * L_ii = sqrt(S_ii - sum_{k<i} L_ik^2).  S is n x n row-major (only its lower
 * triangle is read); L is n x n row-major with zeros above the diagonal.
 * Returns 0, or i + 1 if the pivot of row i is not positive (S is not
 * positive definite). */
int orc_cholesky(const double *S, int n, double *L)
{
    for (size_t k = 0; k < (size_t)n * (size_t)n; ++k) L[k] = 0.0;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = S[(size_t)i * (size_t)n + (size_t)j];
            for (int k = 0; k < j; ++k)
                s -= L[(size_t)i * (size_t)n + (size_t)k] * L[(size_t)j * (size_t)n + (size_t)k];
            if (j < i) {
                L[(size_t)i * (size_t)n + (size_t)j] = s / L[(size_t)j * (size_t)n + (size_t)j];
            } else {
                if (!(s > 0.0)) return i + 1;
                L[(size_t)i * (size_t)n + (size_t)i] = sqrt(s);
            }
        }
    }
    return 0;
}
