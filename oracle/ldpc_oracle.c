/*
 * ldpc_oracle.c - plain, slow CPU oracle for iterative LDPC decoding.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load this library; the decoding library never calls it, and it
 * shares no code, header, table or helper with the CUDA path.
 *
 * What it computes (Amiri & Mehrpouyan, "Multi-Stream LDPC Decoder on GPU of Mobile
 * Devices", arXiv 1812.06545):
 *   - the parity-check matrix H as an edge set between check nodes and variable nodes
 *     (Sec. II, Eq. 1), lifted from a quasi-cyclic base matrix;
 *   - flooding belief propagation / sum-product (Sec. I; Sec. II two-phase message
 *     passing; Algorithm 1 loop order: init, CN->VN, VN->CN, hard decision) in FP64, with
 *     the phi-domain check rule and a clamp on |Q| (the paper gives no formulas; the
 *     textbook rule it cites is written out below);
 *   - horizontal layered decoding (Sec. II, "Algorithm 2": every check of a layer is
 *     computed from the current variable values and those values are updated at once),
 *     with the sum-product rule in FP64 and with normalised min-sum in saturated integer
 *     arithmetic;
 *   - syndrome H.c, dual-diagonal encoding, brute-force maximum-likelihood decoding.
 *
 * Parity pins: every function here is checked by the CPU tests against facts that do
 * not come from this file (hand-derived values, closed forms, brute force, symmetry).
 *
 * Conventions: LLR L = ln P(c=0)/P(c=1); hard decision c = [APP < 0]; sgn(0) = +1;
 * the edges of a check are listed in ascending variable index.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ESTRUCT (-3)

/* ------------------------------------------------------------------ code model */

/* Number of nonzero blocks of a base matrix (entries >= 0), or -1 if an entry is
 * outside [-1, Z). */
int orc_qc_nnz(const int32_t *base, int mb, int nb, int Z)
{
    int nnz = 0;
    for (int i = 0; i < mb * nb; i++) {
        if (base[i] < -1 || base[i] >= Z) return -1;
        if (base[i] >= 0) nnz++;
    }
    return nnz;
}

/* Lift a QC base matrix to H in CSR form (Sec. II: H(i,j) = 1 <=> check i joins
 * variable j).  Check m = l*Z + r of block row l; a block with shift s joins it to
 * variable j*Z + (r + s) mod Z.  rp has mb*Z + 1 entries, ci has nnz*Z. */
int orc_qc_expand(const int32_t *base, int mb, int nb, int Z, int32_t *rp, int32_t *ci)
{
    if (orc_qc_nnz(base, mb, nb, Z) < 0) return ORC_EINVAL;
    int e = 0, m = 0;
    rp[0] = 0;
    for (int l = 0; l < mb; l++) {
        for (int r = 0; r < Z; r++) {
            for (int j = 0; j < nb; j++) {
                int s = base[l * nb + j];
                if (s < 0) continue;
                ci[e++] = j * Z + (r + s) % Z;
            }
            rp[++m] = e;
        }
    }
    return ORC_OK;
}

/* Number of unsatisfied checks of word c under H. */
static int32_t syndrome_weight(int M, const int32_t *rp, const int32_t *ci, const uint8_t *c)
{
    int32_t w = 0;
    for (int m = 0; m < M; m++) {
        int par = 0;
        for (int e = rp[m]; e < rp[m + 1]; e++) par ^= c[ci[e]] & 1;
        w += par;
    }
    return w;
}

int orc_syndrome_batch(int M, int N, const int32_t *rp, const int32_t *ci,
                       const uint8_t *c, int64_t B, int32_t *weight)
{
    for (int64_t b = 0; b < B; b++) weight[b] = syndrome_weight(M, rp, ci, c + b * (int64_t)N);
    return ORC_OK;
}

/* ------------------------------------------------------------------ encoder */

/* Systematic encoding for the dual-diagonal QC recipe by back-substitution over GF(2):
 *   lam_i = sum_{j<kb} P^{s_ij} u_j                  (per block row i)
 *   p_0   = sum_i lam_i                              (the parity column 0 blocks sum to I)
 *   p_1   = lam_0 + P^{s_top} p_0
 *   p_{i+1} = lam_i + p_i + [i == mb/2] P^{s_mid} p_0,  1 <= i <= mb-2
 * and the last block row must close: lam_{mb-1} + P^{s_bot} p_0 + p_{mb-1} = 0.
 * (P^s x)[r] = x[(r + s) mod Z].  Codeword = [u | p_0 .. p_{mb-1}]. */
int orc_encode_qc(const int32_t *base, int mb, int nb, int Z, const uint8_t *u, int64_t B, uint8_t *cw)
{
    int kb = nb - mb, K = kb * Z, N = nb * Z, mid = mb / 2;
    if (mb < 3 || kb < 1 || orc_qc_nnz(base, mb, nb, Z) < 0) return ORC_EINVAL;
    /* structure check */
    for (int i = 0; i < mb; i++) {
        int want = (i == 0 || i == mid || i == mb - 1);
        if ((base[i * nb + kb] >= 0) != want) return ORC_ESTRUCT;
    }
    if (base[0 * nb + kb] != base[(mb - 1) * nb + kb]) return ORC_ESTRUCT;
    for (int c = 1; c < mb; c++)
        for (int i = 0; i < mb; i++) {
            int s = base[i * nb + kb + c];
            int want = (i == c - 1 || i == c);
            if (want ? (s != 0) : (s != -1)) return ORC_ESTRUCT;
        }
    int s_top = base[kb], s_mid = base[mid * nb + kb], s_bot = base[(mb - 1) * nb + kb];
    uint8_t *lam = (uint8_t *)malloc((size_t)mb * Z);
    uint8_t *p = (uint8_t *)malloc((size_t)mb * Z);
    if (!lam || !p) { free(lam); free(p); return ORC_ENOMEM; }
    int rc = ORC_OK;
    for (int64_t b = 0; b < B && rc == ORC_OK; b++) {
        const uint8_t *ub = u + b * (int64_t)K;
        uint8_t *cb = cw + b * (int64_t)N;
        memset(lam, 0, (size_t)mb * Z);
        for (int i = 0; i < mb; i++)
            for (int j = 0; j < kb; j++) {
                int s = base[i * nb + j];
                if (s < 0) continue;
                for (int r = 0; r < Z; r++) lam[i * Z + r] ^= ub[j * Z + (r + s) % Z] & 1;
            }
        for (int r = 0; r < Z; r++) {
            uint8_t acc = 0;
            for (int i = 0; i < mb; i++) acc ^= lam[i * Z + r];
            p[r] = acc;
        }
        for (int r = 0; r < Z; r++) p[1 * Z + r] = lam[r] ^ p[(r + s_top) % Z];
        for (int i = 1; i <= mb - 2; i++)
            for (int r = 0; r < Z; r++) {
                uint8_t v = lam[i * Z + r] ^ p[i * Z + r];
                if (i == mid) v ^= p[(r + s_mid) % Z];
                p[(i + 1) * Z + r] = v;
            }
        for (int r = 0; r < Z; r++)
            if (lam[(mb - 1) * Z + r] ^ p[(r + s_bot) % Z] ^ p[(mb - 1) * Z + r]) rc = ORC_ESTRUCT;
        for (int k = 0; k < K; k++) cb[k] = ub[k] & 1;
        memcpy(cb + K, p, (size_t)mb * Z);
    }
    free(lam);
    free(p);
    return rc;
}

/* ------------------------------------------------------------------ sum-product */

/* phi(x) = -ln tanh(x/2) = ln((e^x + 1)/(e^x - 1)) = log1p(2 / expm1(x)), x > 0. */
static double phi(double x) { return log1p(2.0 / expm1(x)); }

/* Round to the nearest binary16 value, ties to even (used to model messages stored as
 * IEEE half precision).  11 significant bits for |x| >= 2^-14, quantum 2^-24 below,
 * overflow to infinity from 65520 up. */
static double round_binary16(double x)
{
    double a = fabs(x);
    if (a == 0.0 || isnan(x)) return x;
    if (a >= 65520.0) return copysign(INFINITY, x);
    int e;
    frexp(a, &e); /* a = f * 2^e, f in [0.5, 1) */
    int q = e - 11;
    if (q < -24) q = -24;
    double r = nearbyint(ldexp(a, -q));
    return copysign(ldexp(r, q), x);
}

int orc_round_binary16(const double *x, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; i++) out[i] = round_binary16(x[i]);
    return ORC_OK;
}

int orc_phi(const double *x, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; i++) out[i] = phi(x[i]);
    return ORC_OK;
}

static int max_row_degree(int M, const int32_t *rp)
{
    int d = 0;
    for (int m = 0; m < M; m++)
        if (rp[m + 1] - rp[m] > d) d = rp[m + 1] - rp[m];
    return d;
}

static int check_csr(int M, int N, const int32_t *rp, const int32_t *ci)
{
    if (M < 1 || N < 1 || rp[0] != 0) return ORC_EINVAL;
    for (int m = 0; m < M; m++) {
        if (rp[m + 1] - rp[m] < 2) return ORC_EINVAL; /* every check needs >= 2 edges */
        for (int e = rp[m]; e < rp[m + 1]; e++) {
            if (ci[e] < 0 || ci[e] >= N) return ORC_EINVAL;
            if (e > rp[m] && ci[e] <= ci[e - 1]) return ORC_EINVAL; /* ascending, no repeats */
        }
    }
    return ORC_OK;
}

/* Flooding sum-product decoding in FP64 (two-phase message passing, Algorithm 1 order).
 *
 *   init : APP_n = L_n, R_mn = 0
 *   for t = 1..max_iter:
 *     CN : Q_mn = APP_n - R_mn;  for each edge (m,n):
 *          R'_mn = prod_{n' != n} sgn(Q_mn') * min(X, phi( sum_{n' != n} phi(clampX |Q_mn'|) ))
 *          with clampX(x) = min(max(x, phi(X)), X); the exclusive sum and product are
 *          formed directly over the other edges (no total-minus-self).
 *          If fp16_msgs, R' is rounded to binary16 (messages stored in half precision).
 *     VN : APP_n = L_n + sum_m R'_mn;  R <- R'
 *     HD : c_n = [APP_n < 0]
 *     exit: if early_exit and H.c = 0 then iters = t and stop.
 *   Without convergence iters = max_iter and the output is the last hard decision.
 *
 * L: fp32 [B][N] (the same array the GPU decodes); outputs app [B][N] (may be NULL),
 * bits [B][N], iters [B], and the last check-to-variable messages R [B][E] in CSR edge
 * order (may be NULL). */
int orc_spa_flood(int M, int N, const int32_t *rp, const int32_t *ci,
                  const float *L, int64_t B, int max_iter, int early_exit, double X, int fp16_msgs,
                  double *app_out, uint8_t *bits_out, int32_t *iters_out, double *R_out, int nthreads)
{
    if (max_iter < 1 || !(X > 1.0) || check_csr(M, N, rp, ci) != ORC_OK) return ORC_EINVAL;
    const int E = rp[M];
    const int dmax = max_row_degree(M, rp);
    const double phiX = phi(X);
    int rc = ORC_OK;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *app = (double *)malloc(sizeof(double) * N);
        double *R = (double *)malloc(sizeof(double) * E);
        double *Rn = (double *)malloc(sizeof(double) * E);
        double *Q = (double *)malloc(sizeof(double) * dmax);
        uint8_t *hd = (uint8_t *)malloc(N);
        const int ok = app && R && Rn && Q && hd;
        if (!ok) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            rc = ORC_ENOMEM;
        }
        {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int64_t b = 0; b < B; b++) {
                if (!ok) continue;
                const float *Lb = L + b * (int64_t)N;
                for (int n = 0; n < N; n++) app[n] = (double)Lb[n];
                for (int e = 0; e < E; e++) R[e] = 0.0;
                int iters = max_iter;
                for (int t = 1; t <= max_iter; t++) {
                    /* check-node phase */
                    for (int m = 0; m < M; m++) {
                        int e0 = rp[m], dc = rp[m + 1] - rp[m];
                        for (int k = 0; k < dc; k++) Q[k] = app[ci[e0 + k]] - R[e0 + k];
                        for (int k = 0; k < dc; k++) {
                            double sgn = 1.0, sum = 0.0;
                            for (int k2 = 0; k2 < dc; k2++) {
                                if (k2 == k) continue;
                                if (Q[k2] < 0.0) sgn = -sgn;
                                double a = fabs(Q[k2]);
                                if (a < phiX) a = phiX;
                                if (a > X) a = X;
                                sum += phi(a);
                            }
                            double mag = phi(sum);
                            if (mag > X) mag = X;
                            double r = sgn * mag;
                            Rn[e0 + k] = fp16_msgs ? round_binary16(r) : r;
                        }
                    }
                    /* variable-node phase and posterior */
                    for (int e = 0; e < E; e++) R[e] = Rn[e];
                    for (int n = 0; n < N; n++) app[n] = (double)Lb[n];
                    for (int m = 0; m < M; m++)
                        for (int e = rp[m]; e < rp[m + 1]; e++) app[ci[e]] += R[e];
                    /* hard decision and syndrome exit */
                    for (int n = 0; n < N; n++) hd[n] = app[n] < 0.0;
                    if (early_exit && syndrome_weight(M, rp, ci, hd) == 0) {
                        iters = t;
                        break;
                    }
                }
                if (app_out)
                    for (int n = 0; n < N; n++) app_out[b * (int64_t)N + n] = app[n];
                for (int n = 0; n < N; n++) bits_out[b * (int64_t)N + n] = hd[n];
                if (R_out)
                    for (int e = 0; e < E; e++) R_out[b * (int64_t)E + e] = R[e];
                iters_out[b] = iters;
            }
        }
        free(app);
        free(R);
        free(Rn);
        free(Q);
        free(hd);
    }
    return rc;
}

/* ------------------------------------------------------------------ min-sum */

static int32_t sat(int32_t x, int32_t s) { return x > s ? s : (x < -s ? -s : x); }

/* Channel quantiser: q = clamp(rint(s * L), -sat, sat) with one fp32 multiply rounded to
 * nearest and rint rounding half to even. */
int orc_quantize(const float *L, int64_t n, float scale, int satv, int8_t *out)
{
    if (satv < 1 || satv > 127) return ORC_EINVAL;
    for (int64_t i = 0; i < n; i++) {
        volatile float p = scale * L[i]; /* a single fp32 product, no contraction */
        float r = rintf(p);
        int32_t v = r > (float)satv ? satv : (r < -(float)satv ? -satv : (int32_t)r);
        out[i] = (int8_t)v;
    }
    return ORC_OK;
}

/* Layers must be runs of checks that touch pairwise disjoint variables, so that the
 * checks of one layer may be computed in any order (Algorithm 2). */
static int check_layers(int M, int N, const int32_t *rp, const int32_t *ci, int nl, const int32_t *lp)
{
    if (nl < 1 || lp[0] != 0 || lp[nl] != M) return ORC_EINVAL;
    int *seen = (int *)malloc(sizeof(int) * N);
    if (!seen) return ORC_ENOMEM;
    for (int n = 0; n < N; n++) seen[n] = -1;
    int rc = ORC_OK;
    for (int l = 0; l < nl && rc == ORC_OK; l++) {
        if (lp[l + 1] <= lp[l]) rc = ORC_EINVAL;
        for (int m = lp[l]; m < lp[l + 1] && rc == ORC_OK; m++)
            for (int e = rp[m]; e < rp[m + 1]; e++) {
                if (seen[ci[e]] == l) { rc = ORC_EINVAL; break; }
                seen[ci[e]] = l;
            }
    }
    free(seen);
    return rc;
}

/* Horizontal layered sum-product in FP64 (Sec. II "Algorithm 2" schedule with the
 * sum-product check rule of Sec. I): the checks of a layer are computed from the current
 * posteriors, and those posteriors are updated at once.
 *
 *   init : APP_n = L_n, R_mn = 0
 *   for t = 1..max_iter:
 *     for each layer l in order, for each check m of l:
 *       Q_n   = APP_n - R_mn                                      for n in N(m)
 *       R'_mn = prod_{n' != n} sgn(Q_n') * min(X, phi( sum_{n' != n} phi(clampX |Q_n'|) ))
 *               (exclusive sum and product formed directly; rounded to binary16 if fp16_msgs)
 *       APP_n = Q_n + R'_mn;  R_mn <- R'_mn
 *     HD : c_n = [APP_n < 0];  exit as in orc_spa_flood.
 * The check rule, clamp and exit are those of orc_spa_flood; only the schedule differs.
 * Outputs as orc_spa_flood (R_out in CSR edge order, may be NULL). */
int orc_spa_layered(int M, int N, const int32_t *rp, const int32_t *ci, int nl, const int32_t *lp,
                    const float *L, int64_t B, int max_iter, int early_exit, double X, int fp16_msgs,
                    double *app_out, uint8_t *bits_out, int32_t *iters_out, double *R_out, int nthreads)
{
    if (max_iter < 1 || !(X > 1.0) || check_csr(M, N, rp, ci) != ORC_OK) return ORC_EINVAL;
    int lrc = check_layers(M, N, rp, ci, nl, lp);
    if (lrc != ORC_OK) return lrc;
    const int E = rp[M];
    const int dmax = max_row_degree(M, rp);
    const double phiX = phi(X);
    int rc = ORC_OK;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *app = (double *)malloc(sizeof(double) * N);
        double *R = (double *)malloc(sizeof(double) * E);
        double *Q = (double *)malloc(sizeof(double) * dmax);
        double *Rn = (double *)malloc(sizeof(double) * dmax);
        uint8_t *hd = (uint8_t *)malloc(N);
        const int ok = app && R && Q && Rn && hd;
        if (!ok) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            rc = ORC_ENOMEM;
        }
        {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int64_t b = 0; b < B; b++) {
                if (!ok) continue;
                const float *Lb = L + b * (int64_t)N;
                for (int n = 0; n < N; n++) app[n] = (double)Lb[n];
                for (int e = 0; e < E; e++) R[e] = 0.0;
                int iters = max_iter;
                for (int t = 1; t <= max_iter; t++) {
                    for (int l = 0; l < nl; l++) {
                        for (int m = lp[l]; m < lp[l + 1]; m++) {
                            int e0 = rp[m], dc = rp[m + 1] - rp[m];
                            for (int k = 0; k < dc; k++) Q[k] = app[ci[e0 + k]] - R[e0 + k];
                            for (int k = 0; k < dc; k++) {
                                double sgn = 1.0, sum = 0.0;
                                for (int k2 = 0; k2 < dc; k2++) {
                                    if (k2 == k) continue;
                                    if (Q[k2] < 0.0) sgn = -sgn;
                                    double a = fabs(Q[k2]);
                                    if (a < phiX) a = phiX;
                                    if (a > X) a = X;
                                    sum += phi(a);
                                }
                                double mag = phi(sum);
                                if (mag > X) mag = X;
                                double r = sgn * mag;
                                Rn[k] = fp16_msgs ? round_binary16(r) : r;
                            }
                            for (int k = 0; k < dc; k++) {
                                R[e0 + k] = Rn[k];
                                app[ci[e0 + k]] = Q[k] + Rn[k];
                            }
                        }
                    }
                    for (int n = 0; n < N; n++) hd[n] = app[n] < 0.0;
                    if (early_exit && syndrome_weight(M, rp, ci, hd) == 0) {
                        iters = t;
                        break;
                    }
                }
                if (app_out)
                    for (int n = 0; n < N; n++) app_out[b * (int64_t)N + n] = app[n];
                for (int n = 0; n < N; n++) bits_out[b * (int64_t)N + n] = hd[n];
                if (R_out)
                    for (int e = 0; e < E; e++) R_out[b * (int64_t)E + e] = R[e];
                iters_out[b] = iters;
            }
        }
        free(app);
        free(R);
        free(Q);
        free(Rn);
        free(hd);
    }
    return rc;
}

/* Horizontal layered normalised min-sum in saturated integer arithmetic.
 *
 *   init : APP_n = q_n (channel LLRs already quantised), R_mn = 0
 *   for t = 1..max_iter:
 *     for each layer l in order, for each check m of l:
 *       Q_n   = sat(APP_n - R_mn, msg_sat)                  for n in N(m)
 *       min1  = min |Q_n|, min2 = second smallest |Q_n| (duplicates counted),
 *       S     = XOR of [Q_n < 0]
 *       mag_n = min2 for the first edge attaining min1, else min1
 *               (if two edges tie at min1 then min2 = min1, so the choice is immaterial)
 *       R_mn  = (S xor [Q_n < 0]) ? -((alpha_num*mag_n) >> alpha_shift)
 *                                 :  ((alpha_num*mag_n) >> alpha_shift)
 *       APP_n = sat(Q_n + R_mn, app_sat)
 *     HD : c_n = [APP_n < 0];  exit as in orc_spa_flood.
 * All arithmetic in int32; saturation only at the two points shown. */
int orc_nms_layered(int M, int N, const int32_t *rp, const int32_t *ci, int nl, const int32_t *lp,
                    const int8_t *q, int64_t B, int max_iter, int early_exit,
                    int alpha_num, int alpha_shift, int msg_sat, int app_sat,
                    int32_t *app_out, uint8_t *bits_out, int32_t *iters_out, int nthreads)
{
    if (max_iter < 1 || alpha_num < 1 || alpha_shift < 0 || alpha_shift > 16 || msg_sat < 1 || app_sat < msg_sat)
        return ORC_EINVAL;
    if (check_csr(M, N, rp, ci) != ORC_OK) return ORC_EINVAL;
    int lrc = check_layers(M, N, rp, ci, nl, lp);
    if (lrc != ORC_OK) return lrc;
    const int E = rp[M];
    const int dmax = max_row_degree(M, rp);
    int rc = ORC_OK;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        int32_t *app = (int32_t *)malloc(sizeof(int32_t) * N);
        int32_t *R = (int32_t *)malloc(sizeof(int32_t) * E);
        int32_t *Q = (int32_t *)malloc(sizeof(int32_t) * dmax);
        uint8_t *hd = (uint8_t *)malloc(N);
        const int ok = app && R && Q && hd;
        if (!ok) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            rc = ORC_ENOMEM;
        }
        {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
            for (int64_t b = 0; b < B; b++) {
                if (!ok) continue;
                const int8_t *qb = q + b * (int64_t)N;
                for (int n = 0; n < N; n++) app[n] = qb[n];
                for (int e = 0; e < E; e++) R[e] = 0;
                int iters = max_iter;
                for (int t = 1; t <= max_iter; t++) {
                    for (int l = 0; l < nl; l++) {
                        for (int m = lp[l]; m < lp[l + 1]; m++) {
                            int e0 = rp[m], dc = rp[m + 1] - rp[m];
                            int32_t min1 = INT32_MAX, min2 = INT32_MAX, S = 0, arg = -1;
                            for (int k = 0; k < dc; k++) {
                                Q[k] = sat(app[ci[e0 + k]] - R[e0 + k], msg_sat);
                                int32_t a = Q[k] < 0 ? -Q[k] : Q[k];
                                if (a < min1) {
                                    min2 = min1;
                                    min1 = a;
                                    arg = k;
                                } else if (a < min2) {
                                    min2 = a;
                                }
                                S ^= (Q[k] < 0);
                            }
                            for (int k = 0; k < dc; k++) {
                                int32_t mag = (k == arg) ? min2 : min1;
                                int32_t magp = (alpha_num * mag) >> alpha_shift;
                                int32_t neg = S ^ (Q[k] < 0);
                                R[e0 + k] = neg ? -magp : magp;
                                app[ci[e0 + k]] = sat(Q[k] + R[e0 + k], app_sat);
                            }
                        }
                    }
                    for (int n = 0; n < N; n++) hd[n] = app[n] < 0;
                    if (early_exit && syndrome_weight(M, rp, ci, hd) == 0) {
                        iters = t;
                        break;
                    }
                }
                if (app_out)
                    for (int n = 0; n < N; n++) app_out[b * (int64_t)N + n] = app[n];
                for (int n = 0; n < N; n++) bits_out[b * (int64_t)N + n] = hd[n];
                iters_out[b] = iters;
            }
        }
        free(app);
        free(R);
        free(Q);
        free(hd);
    }
    return rc;
}

/* The same layered normalised min-sum written in real arithmetic with no saturation:
 * R_mn = sgn * floor(alpha * mag) with mag taken from the other edges' |Q| by a direct
 * minimum over n' != n.  A second, plainer statement of the check rule used to cross-check
 * the integer routine where no saturation occurs. */
int orc_nms_layered_real(int M, int N, const int32_t *rp, const int32_t *ci, int nl, const int32_t *lp,
                         const double *L, int64_t B, int max_iter, double alpha,
                         double *app_out, int nthreads)
{
    (void)nthreads;
    if (max_iter < 1 || check_csr(M, N, rp, ci) != ORC_OK) return ORC_EINVAL;
    int lrc = check_layers(M, N, rp, ci, nl, lp);
    if (lrc != ORC_OK) return lrc;
    const int E = rp[M];
    const int dmax = max_row_degree(M, rp);
    double *app = (double *)malloc(sizeof(double) * N);
    double *R = (double *)calloc(E, sizeof(double));
    double *Q = (double *)malloc(sizeof(double) * dmax);
    if (!app || !R || !Q) { free(app); free(R); free(Q); return ORC_ENOMEM; }
    for (int64_t b = 0; b < B; b++) {
        for (int n = 0; n < N; n++) app[n] = L[b * (int64_t)N + n];
        for (int e = 0; e < E; e++) R[e] = 0.0;
        for (int t = 1; t <= max_iter; t++)
            for (int l = 0; l < nl; l++)
                for (int m = lp[l]; m < lp[l + 1]; m++) {
                    int e0 = rp[m], dc = rp[m + 1] - rp[m];
                    for (int k = 0; k < dc; k++) Q[k] = app[ci[e0 + k]] - R[e0 + k];
                    for (int k = 0; k < dc; k++) {
                        double mn = INFINITY, sgn = 1.0;
                        for (int k2 = 0; k2 < dc; k2++) {
                            if (k2 == k) continue;
                            if (fabs(Q[k2]) < mn) mn = fabs(Q[k2]);
                            if (Q[k2] < 0.0) sgn = -sgn;
                        }
                        R[e0 + k] = sgn * floor(alpha * mn);
                    }
                    for (int k = 0; k < dc; k++) app[ci[e0 + k]] = Q[k] + R[e0 + k];
                }
        for (int n = 0; n < N; n++) app_out[b * (int64_t)N + n] = app[n];
    }
    free(app);
    free(R);
    free(Q);
    return ORC_OK;
}

/* ------------------------------------------------------------------ ML */

/* Brute-force maximum-likelihood decoding for N <= 24: enumerate every word x in
 * [0, 2^N), keep those with H.x = 0, and return argmax_c sum_n (1 - 2 c_n) L_n
 * (first maximiser in enumeration order).  Bit n of x is codeword bit n. */
int orc_ml_decode(int M, int N, const int32_t *rp, const int32_t *ci,
                  const float *L, int64_t B, uint8_t *bits_out, int32_t *codebook_size)
{
    if (N < 1 || N > 24 || check_csr(M, N, rp, ci) != ORC_OK) return ORC_EINVAL;
    uint32_t *rowmask = (uint32_t *)calloc(M, sizeof(uint32_t));
    if (!rowmask) return ORC_ENOMEM;
    for (int m = 0; m < M; m++)
        for (int e = rp[m]; e < rp[m + 1]; e++) rowmask[m] |= 1u << ci[e];
    uint32_t ncw = 0, cap = 1024;
    uint32_t *cb = (uint32_t *)malloc(sizeof(uint32_t) * cap);
    if (!cb) { free(rowmask); return ORC_ENOMEM; }
    for (uint32_t x = 0; x < (1u << N); x++) {
        int ok = 1;
        for (int m = 0; m < M && ok; m++) ok = (__builtin_popcount(x & rowmask[m]) & 1) == 0;
        if (!ok) continue;
        if (ncw == cap) {
            cap *= 2;
            uint32_t *nb2 = (uint32_t *)realloc(cb, sizeof(uint32_t) * cap);
            if (!nb2) { free(cb); free(rowmask); return ORC_ENOMEM; }
            cb = nb2;
        }
        cb[ncw++] = x;
    }
    if (codebook_size) *codebook_size = (int32_t)ncw;
    for (int64_t b = 0; b < B; b++) {
        const float *Lb = L + b * (int64_t)N;
        double best = -INFINITY;
        uint32_t arg = 0;
        for (uint32_t i = 0; i < ncw; i++) {
            double corr = 0.0;
            for (int n = 0; n < N; n++) corr += ((cb[i] >> n) & 1u) ? -(double)Lb[n] : (double)Lb[n];
            if (corr > best) { best = corr; arg = cb[i]; }
        }
        for (int n = 0; n < N; n++) bits_out[b * (int64_t)N + n] = (arg >> n) & 1u;
    }
    free(cb);
    free(rowmask);
    return ORC_OK;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
